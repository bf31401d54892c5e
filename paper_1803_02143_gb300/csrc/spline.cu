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
#include <algorithm>

#include "ctx.h"
#include "sweep_kernels.cuh"

namespace sldg {

namespace {

constexpr int kSplLines = 32;
constexpr int kSplChunks = 4;
constexpr int kSplThreads = kSplLines * kSplChunks;
constexpr int kSplPitch = kSplLines + 1;
constexpr int kSplRegPts = 32;  // chunk points held in registers (RC)

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
// (block / key_div) % key_mod.  A CTA walks tiles tile0, tile0 + gridDim.x,
// ...: with NB = 2 the next tile is staged by cp.async into the second
// input buffer while the current one is computed (NB = 1: each tile is
// staged after the previous one, the overlap coming from the other CTAs
// on the SM).  RC (FP64 chunks of at most kSplRegPts points): a thread keeps its
// chunk of y in registers from the causal recurrence to the anti-causal
// one, and across a strided direction (a warp's lanes on 32 consecutive
// columns) writes the interpolant straight to f, coalesced, instead of
// through the tile.
template <typename T, bool CONTIG, bool KEYCOL, int NB, bool RC>
__global__ void __launch_bounds__(kSplThreads)
    k_spline_sweep(T* __restrict__ f, int n, long long inner, long long outer,
                   long long tiles_per_block, long long ntiles, const T* __restrict__ theta,
                   const int* __restrict__ svec, long long key_div, long long key_mod, T z,
                   int W) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* Ubuf = reinterpret_cast<T*>(smraw);     // two input buffers [n][kSplPitch]
  T* Y = Ubuf + NB * (size_t)n * kSplPitch;  // [n][kSplPitch]
  const int tid = threadIdx.x;
  const int warp = tid / kSplLines, lane = tid % kSplLines;
  constexpr int kWarps = kSplThreads / kSplLines;
  struct Tile {
    long long b0, j0;  // first line: block, column
    int nl;            // lines of this tile
  };
  auto tile_of = [&](long long t) {
    Tile x;
    if (CONTIG) {
      x.b0 = t * kSplLines;
      x.j0 = 0;
      x.nl = (int)min((long long)kSplLines, outer - x.b0);
    } else {
      x.b0 = t / tiles_per_block;
      x.j0 = (t - x.b0 * tiles_per_block) * kSplLines;
      x.nl = (int)min((long long)kSplLines, inner - x.j0);
    }
    return x;
  };
  auto base_of = [&](const Tile& x) {
    return CONTIG ? f + x.b0 * n : f + x.b0 * n * inner + x.j0;
  };
  // staging: every read coalesced (a warp along a line, or along a row of
  // the column tile); the padded pitch keeps the transposed writes free of
  // bank conflicts
  auto stage = [&](const Tile& x, T* U) {
    const T* base = base_of(x);
    if (CONTIG) {
      for (int l = warp; l < x.nl; l += kWarps) {
        const T* src = base + (long long)l * n;
        for (int i = lane; i < n; i += kSplLines)
          cp_async_elem<sizeof(T)>(U + i * kSplPitch + l, src + i);
      }
    } else if (lane < x.nl) {
      for (int i = warp; i < n; i += kWarps)
        cp_async_elem<sizeof(T)>(U + i * kSplPitch + lane, base + (long long)i * inner + lane);
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };

  const int l = tid % kSplLines, c = tid / kSplLines;
  const int C = (n + kSplChunks - 1) / kSplChunks;
  const int ib = min(c * C, n), ie = min(ib + C, n);
  long long t = blockIdx.x;
  if (NB == 2 && t < ntiles) stage(tile_of(t), Ubuf);
  for (int b = 0; t < ntiles; t += gridDim.x, b ^= 1) {
    const Tile x = tile_of(t);
    T* U = Ubuf + (size_t)(NB == 2 ? b : 0) * n * kSplPitch;
    if (NB == 1) stage(x, U);  // the previous tile's reads of U ended at its last barrier
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    __syncthreads();  // this tile staged; the other buffer and Y are free
    if (NB == 2 && t + gridDim.x < ntiles)
      stage(tile_of(t + gridDim.x), Ubuf + (size_t)(b ^ 1) * n * kSplPitch);
    const bool act = l < x.nl && ib < ie;
    T* Ul = U + l;
    T* Yl = Y + l;
    // The recurrences run eight points at a time: the eight shared-memory
    // loads of a batch are issued before its chain of dependent FMAs.
    constexpr int B8 = 8;
    T yr[RC ? kSplRegPts : 1];  // the chunk's y (RC)
    // causal recurrence y_i = u_i - z y_{i-1}: W warm-up points (a multiple
    // of 8) from zero, then the chunk ib .. ie - 1 into Y
    if (act) {
      T y = T(0);
      int k = (ib - W) % n;
      if (k < 0) k += n;
      for (int q0 = 0; q0 < W; q0 += B8) {
        T u[B8];
#pragma unroll
        for (int q = 0; q < B8; ++q) {
          u[q] = Ul[k * kSplPitch];
          k = k + 1 == n ? 0 : k + 1;
        }
#pragma unroll
        for (int q = 0; q < B8; ++q) y = fma(-z, y, u[q]);
      }
      if constexpr (RC) {
        const int len = ie - ib;
#pragma unroll
        for (int q0 = 0; q0 < kSplRegPts; q0 += B8) {
          T u[B8];
#pragma unroll
          for (int q = 0; q < B8; ++q)
            if (q0 + q < len) u[q] = Ul[(ib + q0 + q) * kSplPitch];
#pragma unroll
          for (int q = 0; q < B8; ++q)
            if (q0 + q < len) {
              y = fma(-z, y, u[q]);
              yr[q0 + q] = y;
              Yl[(ib + q0 + q) * kSplPitch] = y;  // for the neighbours' warm-up
            }
        }
      } else {
        int i = ib;
        for (; i + B8 <= ie; i += B8) {
          T u[B8];
#pragma unroll
          for (int q = 0; q < B8; ++q) u[q] = Ul[(i + q) * kSplPitch];
#pragma unroll
          for (int q = 0; q < B8; ++q) {
            y = fma(-z, y, u[q]);
            Yl[(i + q) * kSplPitch] = y;
          }
        }
        for (; i < ie; ++i) {
          y = fma(-z, y, Ul[i * kSplPitch]);
          Yl[i * kSplPitch] = y;
        }
      }
    }
    __syncthreads();
    // anti-causal recurrence v_i = y_i - z v_{i+1}; w = 6 z v over u
    if (act) {
      T v = T(0);
      int k = (ie - 1 + W) % n;
      for (int q0 = 0; q0 < W; q0 += B8) {
        T u[B8];
#pragma unroll
        for (int q = 0; q < B8; ++q) {
          u[q] = Yl[k * kSplPitch];
          k = k == 0 ? n - 1 : k - 1;
        }
#pragma unroll
        for (int q = 0; q < B8; ++q) v = fma(-z, v, u[q]);
      }
      const T sz = T(6) * z;
      if constexpr (RC) {
        const int len = ie - ib;
#pragma unroll
        for (int q = kSplRegPts - 1; q >= 0; --q)
          if (q < len) {
            v = fma(-z, v, yr[q]);
            Ul[(ib + q) * kSplPitch] = sz * v;
          }
      } else {
        int i = ie - 1;
        for (; i - B8 + 1 >= ib; i -= B8) {
          T u[B8];
#pragma unroll
          for (int q = 0; q < B8; ++q) u[q] = Yl[(i - q) * kSplPitch];
#pragma unroll
          for (int q = 0; q < B8; ++q) {
            v = fma(-z, v, u[q]);
            Ul[(i - q) * kSplPitch] = sz * v;
          }
        }
        for (; i >= ib; --i) {
          v = fma(-z, v, Yl[i * kSplPitch]);
          Ul[i * kSplPitch] = sz * v;
        }
      }
    }
    __syncthreads();
    // the interpolant at the shifted points
    if (act) {
      const long long key = KEYCOL ? (x.j0 + l) % key_mod
                                   : ((CONTIG ? x.b0 + l : x.b0) / key_div) % key_mod;
      const T th = theta[key];
      const int s = svec[key];
      const T om = T(1) - th, sixth = T(1) / T(6);
      const T w0 = th * th * th * sixth;
      const T w1 = (T(4) - T(6) * om * om + T(3) * om * om * om) * sixth;
      const T w2 = (T(4) - T(6) * th * th + T(3) * th * th * th) * sixth;
      const T w3 = om * om * om * sixth;
      // output point i: the tile's Y, or (RC across a strided direction) f
      constexpr bool DIRECT = RC && !CONTIG;
      T* const orow = DIRECT ? base_of(x) + l : Yl;
      const long long ostr = DIRECT ? inner : kSplPitch;
      int k = (ib - s - 2) % n;
      if (k < 0) k += n;
      T c0 = Ul[k * kSplPitch];
      k = k + 1 == n ? 0 : k + 1;
      T c1 = Ul[k * kSplPitch];
      k = k + 1 == n ? 0 : k + 1;
      T c2 = Ul[k * kSplPitch];
      k = k + 1 == n ? 0 : k + 1;
      int i = ib;
      for (; i + B8 <= ie; i += B8) {
        T u[B8];
#pragma unroll
        for (int q = 0; q < B8; ++q) {
          u[q] = Ul[k * kSplPitch];
          k = k + 1 == n ? 0 : k + 1;
        }
#pragma unroll
        for (int q = 0; q < B8; ++q) {
          orow[(i + q) * ostr] = fma(w0, c0, fma(w1, c1, fma(w2, c2, w3 * u[q])));
          c0 = c1;
          c1 = c2;
          c2 = u[q];
        }
      }
      for (; i < ie; ++i) {
        const T c3 = Ul[k * kSplPitch];
        k = k + 1 == n ? 0 : k + 1;
        orow[i * ostr] = fma(w0, c0, fma(w1, c1, fma(w2, c2, w3 * c3)));
        c0 = c1;
        c1 = c2;
        c2 = c3;
      }
    }
    __syncthreads();  // (the next tile may then be staged into U)
    if (RC && !CONTIG) continue;  // written by the evaluation
    T* base = base_of(x);
    if (CONTIG) {
      for (int ll = warp; ll < x.nl; ll += kWarps) {
        T* dst = base + (long long)ll * n;
        for (int i = lane; i < n; i += kSplLines) dst[i] = Y[i * kSplPitch + ll];
      }
    } else if (lane < x.nl) {
      for (int i = warp; i < n; i += kWarps)
        base[(long long)i * inner + lane] = Y[i * kSplPitch + lane];
    }
  }
}

template <typename T, bool CONTIG, bool KEYCOL>
cudaError_t launch_spline_T(const SweepArgs& a, cudaStream_t st) {
  const int n = a.nc;
  const size_t buf = (size_t)n * kSplPitch * sizeof(T);
  if (n < 3 || 2 * buf > 227 * 1024) return cudaErrorNotSupported;
  // two input buffers only where they cost no CTA (eight per SM still fit):
  // at 128 points one buffer and more CTAs (six per SM in FP32, three in
  // FP64) beat two buffers (four, two): 0.573 against 0.602 ms per FP32
  // v-sweep and 4.88 against 5.12 ms per FP64 v-sweep at 128^4 points
  const int nb = 8 * (3 * buf + 1024) <= 228 * 1024 ? 2 : 1;
  const size_t smem = (nb + 1) * buf;
  // FP64 chunks of at most kSplRegPts points stay in registers (at 128^4
  // points 4.71 against 4.87 ms per v-sweep, 9.49 against 10.11 per pair of
  // x1 sweeps); FP32 gains nothing from it (0.578 against 0.573 ms)
  const bool rc = sizeof(T) == 8 && (n + kSplChunks - 1) / kSplChunks <= kSplRegPts;
  auto kfn = nb == 2 ? (rc ? k_spline_sweep<T, CONTIG, KEYCOL, 2, true> : k_spline_sweep<T, CONTIG, KEYCOL, 2, false>)
                     : (rc ? k_spline_sweep<T, CONTIG, KEYCOL, 1, true> : k_spline_sweep<T, CONTIG, KEYCOL, 1, false>);
  if (smem > 48 * 1024) {
    const cudaError_t e =
        cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const long long tiles_per_block = CONTIG ? 1 : (a.inner + kSplLines - 1) / kSplLines;
  const long long ntiles = CONTIG ? (a.outer + kSplLines - 1) / kSplLines : a.outer * tiles_per_block;
  // persistent CTAs: as many as are resident at once (by shared memory,
  // at most 8 per SM), each walking tiles with a stride of the grid
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const long long per_sm = std::max<long long>(1, std::min<long long>(8, (228 * 1024) / (smem + 1024)));
  const long long blocks = std::min<long long>(ntiles, per_sm * sms);
  if (blocks < 1) return cudaSuccess;
  const T z = T(2.0 - 1.7320508075688772);  // 2 - sqrt(3)
  const int W = sizeof(T) == 8 ? 32 : 16;
  kfn<<<(unsigned)blocks, kSplThreads, smem, st>>>(
      static_cast<T*>(a.f), n, a.inner, a.outer, tiles_per_block, ntiles,
      static_cast<const T*>(a.ab), a.s, a.key_div, a.key_mod, z, W);
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
