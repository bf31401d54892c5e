// sweep_kernels.cuh -- the SLDG sweep kernels: one 1D projected translation
// (Eq. (AB-sldg)) applied in place to every line of f along one direction,
// and its transpose.
//
// Forward, target cell c of a line with integer shift s:
//   out[c] = A in[c-s-1] + B in[c-s]          (i* = c-s-1, i*+1 = c-s)
// Transpose (adjoint), source cell c:
//   in_bar[c] = A^T out_bar[c+s+1] + B^T out_bar[c+s]
// Source cells wrap (periodic x, or periodic-v test mode) or are dropped
// (zero inflow in v).
//
// Each CTA stages whole lines in shared memory before writing any output,
// so the update is in place: every line is owned by exactly one CTA and is
// read completely before the first store to it.
#pragma once

#include <type_traits>

#include "ctx.h"

namespace sldg {

constexpr int kStridedW = 32;       // columns per tile of a strided sweep
constexpr int kStridedThreads = 256;
constexpr int kStridedGroups = kStridedThreads / kStridedW;
constexpr int kX1Threads = 256;

// ---------------------------------------------------------------------------
// Strided sweep (x2, v1, v2): f viewed as [outer][D][inner]; a tile is one
// outer index and kStridedW consecutive inner columns, all D rows.
//   PERCOL: matrix key per column (v-sweeps: key = column % key_mod, the
//           x-node); else per tile (x2-sweep: key = (outer / key_div) % key_mod).
//   EBAR:   also accumulate d/dE <out_bar, S(E) g> per column into epart
//           (adjoint v-sweeps); g is the forward input of the sweep.
// ---------------------------------------------------------------------------
template <typename T, int N, bool PERIODIC, bool PERCOL, bool ADJ, bool EBAR>
__global__ void __launch_bounds__(kStridedThreads)
    k_sweep_strided(T* __restrict__ f, const T* __restrict__ gfwd, double* __restrict__ epart,
                    long long inner, int nc, long long ncolblk, const T* __restrict__ ab,
                    const T* __restrict__ dab, const int* __restrict__ svec, long long mcount,
                    long long key_div, long long key_mod) {
  constexpr int W = kStridedW, G = kStridedGroups;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* tile = reinterpret_cast<T*>(smraw);
  const int D = nc * N;
  const long long cb = blockIdx.x % ncolblk;
  const long long o = blockIdx.x / ncolblk;
  const int lane = threadIdx.x & (W - 1);
  const int grp = threadIdx.x / W;
  const long long col0 = cb * W;
  const long long col = col0 + lane;
  const bool valid = col < inner;
  const long long base = o * (long long)D * inner + col0;
  T* fb = f + base;

#pragma unroll 4
  for (int r = grp; r < D; r += G) tile[r * W + lane] = valid ? fb[(long long)r * inner + lane] : T(0);
  __syncthreads();

  double eacc = 0.0;
  if (valid) {
    const long long key = PERCOL ? (col % key_mod) : ((o / key_div) % key_mod);
    T A[N * N], B[N * N];
#pragma unroll
    for (int i = 0; i < N * N; ++i) {
      A[i] = ab[(long long)i * mcount + key];
      B[i] = ab[(long long)(N * N + i) * mcount + key];
    }
    const int s = svec[key];
    for (int c = grp; c < nc; c += G) {
      int ka = ADJ ? c + s + 1 : c - s - 1;
      int kb = ADJ ? c + s : c - s;
      bool va = true, vb = true;
      if (PERIODIC) {
        ka = wrap_cell(ka, nc);
        kb = wrap_cell(kb, nc);
      } else {
        va = ka >= 0 && ka < nc;
        vb = kb >= 0 && kb < nc;
      }
      T xa[N], xb[N];
#pragma unroll
      for (int l = 0; l < N; ++l) {
        xa[l] = va ? tile[(ka * N + l) * W + lane] : T(0);
        xb[l] = vb ? tile[(kb * N + l) * W + lane] : T(0);
      }
#pragma unroll
      for (int j = 0; j < N; ++j) {
        T acc = T(0);
#pragma unroll
        for (int l = 0; l < N; ++l) {
          acc = fma(ADJ ? A[l * N + j] : A[j * N + l], xa[l], acc);
          acc = fma(ADJ ? B[l * N + j] : B[j * N + l], xb[l], acc);
        }
        fb[(long long)(c * N + j) * inner + lane] = acc;
      }
    }
    if (EBAR) {
      // d/dtheta of <lam_out, S g>: lam_out[c] is the staged tile, g at the
      // forward source cells c-s-1, c-s.
      T dA[N * N], dB[N * N];
#pragma unroll
      for (int i = 0; i < N * N; ++i) {
        dA[i] = dab[(long long)i * mcount + key];
        dB[i] = dab[(long long)(N * N + i) * mcount + key];
      }
      const T* gb = gfwd + base;
      for (int c = grp; c < nc; c += G) {
        int ka = c - s - 1, kb = c - s;
        bool va = true, vb = true;
        if (PERIODIC) {
          ka = wrap_cell(ka, nc);
          kb = wrap_cell(kb, nc);
        } else {
          va = ka >= 0 && ka < nc;
          vb = kb >= 0 && kb < nc;
        }
        T ga[N], gbv[N];
#pragma unroll
        for (int l = 0; l < N; ++l) {
          ga[l] = va ? gb[(long long)(ka * N + l) * inner + lane] : T(0);
          gbv[l] = vb ? gb[(long long)(kb * N + l) * inner + lane] : T(0);
        }
        T cell = T(0);
#pragma unroll
        for (int j = 0; j < N; ++j) {
          T d = T(0);
#pragma unroll
          for (int l = 0; l < N; ++l) {
            d = fma(dA[j * N + l], ga[l], d);
            d = fma(dB[j * N + l], gbv[l], d);
          }
          cell = fma(tile[(c * N + j) * W + lane], d, cell);
        }
        eacc += (double)cell;
      }
    }
  }
  if (EBAR) {
    // reduce the kStridedGroups partial sums of each column in a fixed order
    __syncthreads();
    double* red = reinterpret_cast<double*>(smraw);
    red[grp * W + lane] = eacc;
    __syncthreads();
    if (grp == 0 && valid) {
      double t = 0.0;
#pragma unroll
      for (int q = 0; q < G; ++q) t += red[q * W + lane];
      epart[o * inner + col] = t;
    }
  }
}

// ---------------------------------------------------------------------------
// x1-sweep: lines are contiguous; a tile is R consecutive lines (R divides
// D1, so all lines of a tile share their v1 node and matrices).  Input and
// output are staged in shared memory, loads and stores are contiguous.
// ---------------------------------------------------------------------------
template <typename T, int N, bool ADJ>
__global__ void __launch_bounds__(kX1Threads)
    k_sweep_x1(T* __restrict__ f, int nc, int R, const T* __restrict__ ab,
               const int* __restrict__ svec, long long mcount, long long key_div,
               long long key_mod) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int D = nc * N;
  const int TL = R * D;
  const int TLp = (TL + 3) & ~3;  // keep the output buffer 16-byte aligned
  T* sin = reinterpret_cast<T*>(smraw);
  T* sout = sin + TLp;
  const long long t0 = (long long)blockIdx.x * TL;
  T* fb = f + t0;
  constexpr int V = 16 / sizeof(T);  // elements per 16-byte vector
  const bool vec = (TL % V == 0) && ((reinterpret_cast<uintptr_t>(fb) & 15) == 0);
  if (vec) {
    using V4 = typename std::conditional<sizeof(T) == 8, double2, float4>::type;
    const V4* src = reinterpret_cast<const V4*>(fb);
    V4* dst = reinterpret_cast<V4*>(sin);
    for (int i = threadIdx.x; i < TL / V; i += blockDim.x) dst[i] = src[i];
  } else {
    for (int i = threadIdx.x; i < TL; i += blockDim.x) sin[i] = fb[i];
  }
  __syncthreads();

  const long long L0 = (long long)blockIdx.x * R;
  const long long key = (L0 / key_div) % key_mod;
  T A[N * N], B[N * N];
#pragma unroll
  for (int i = 0; i < N * N; ++i) {
    A[i] = ab[(long long)i * mcount + key];
    B[i] = ab[(long long)(N * N + i) * mcount + key];
  }
  const int s = svec[key];
  for (int idx = threadIdx.x; idx < R * nc; idx += blockDim.x) {
    const int r = idx / nc, c = idx - r * nc;
    const int ka = wrap_cell(ADJ ? c + s + 1 : c - s - 1, nc);
    const int kb = wrap_cell(ADJ ? c + s : c - s, nc);
    const T* row = sin + r * D;
    T xa[N], xb[N];
#pragma unroll
    for (int l = 0; l < N; ++l) {
      xa[l] = row[ka * N + l];
      xb[l] = row[kb * N + l];
    }
#pragma unroll
    for (int j = 0; j < N; ++j) {
      T acc = T(0);
#pragma unroll
      for (int l = 0; l < N; ++l) {
        acc = fma(ADJ ? A[l * N + j] : A[j * N + l], xa[l], acc);
        acc = fma(ADJ ? B[l * N + j] : B[j * N + l], xb[l], acc);
      }
      sout[r * D + c * N + j] = acc;
    }
  }
  __syncthreads();
  if (vec) {
    using V4 = typename std::conditional<sizeof(T) == 8, double2, float4>::type;
    const V4* src = reinterpret_cast<const V4*>(sout);
    V4* dst = reinterpret_cast<V4*>(fb);
    for (int i = threadIdx.x; i < TL / V; i += blockDim.x) dst[i] = src[i];
  } else {
    for (int i = threadIdx.x; i < TL; i += blockDim.x) fb[i] = sout[i];
  }
}

inline size_t strided_smem(size_t esize, long long D) {
  size_t t = (size_t)D * kStridedW * esize;
  size_t r = (size_t)kStridedThreads * sizeof(double);  // EBAR reduction reuse
  return t > r ? t : r;
}

inline size_t x1_smem(size_t esize, long long D, int R) {
  size_t TL = (size_t)R * (size_t)D;
  size_t TLp = (TL + 3) & ~(size_t)3;
  return (TLp + TL) * esize;
}

template <typename T, int N>
cudaError_t launch_sweep_T(const SweepArgs& a, cudaStream_t st) {
  T* f = reinterpret_cast<T*>(a.f);
  const T* ab = reinterpret_cast<const T*>(a.ab);
  const T* dab = reinterpret_cast<const T*>(a.dab);
  const long long D = (long long)a.nc * N;
  if (a.dim == 0) {
    const int R = a.lines_per_tile;
    const long long nlines = a.outer;  // for x1, outer = number of lines
    const long long tiles = nlines / R;
    const size_t smem = x1_smem(sizeof(T), D, R);
    auto kfn = a.adjoint ? k_sweep_x1<T, N, true> : k_sweep_x1<T, N, false>;
    if (smem > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    kfn<<<(unsigned)tiles, kX1Threads, smem, st>>>(f, a.nc, R, ab, a.s, a.mcount, a.key_div,
                                                   a.key_mod);
    return cudaGetLastError();
  }
  const long long ncolblk = (a.inner + kStridedW - 1) / kStridedW;
  const long long blocks = ncolblk * a.outer;
  const size_t smem = strided_smem(sizeof(T), D);
  const T* g = reinterpret_cast<const T*>(a.g);
  decltype(&k_sweep_strided<T, N, true, false, false, false>) kfn;
  const bool percol = a.dim >= 2;
  const bool ebar = a.adjoint && percol && a.g != nullptr && a.epart != nullptr;
  if (!percol) {
    kfn = a.adjoint ? k_sweep_strided<T, N, true, false, true, false>
                    : k_sweep_strided<T, N, true, false, false, false>;
  } else if (a.periodic) {
    if (!a.adjoint) kfn = k_sweep_strided<T, N, true, true, false, false>;
    else kfn = ebar ? k_sweep_strided<T, N, true, true, true, true>
                    : k_sweep_strided<T, N, true, true, true, false>;
  } else {
    if (!a.adjoint) kfn = k_sweep_strided<T, N, false, true, false, false>;
    else kfn = ebar ? k_sweep_strided<T, N, false, true, true, true>
                    : k_sweep_strided<T, N, false, true, true, false>;
  }
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  kfn<<<(unsigned)blocks, kStridedThreads, smem, st>>>(f, g, a.epart, a.inner, a.nc, ncolblk, ab,
                                                       dab, a.s, a.mcount, a.key_div, a.key_mod);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_sweep_any(const SweepArgs& a, cudaStream_t st) {
  switch (a.n) {
    case 1: return launch_sweep_T<T, 1>(a, st);
    case 2: return launch_sweep_T<T, 2>(a, st);
    case 3: return launch_sweep_T<T, 3>(a, st);
    case 4: return launch_sweep_T<T, 4>(a, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace sldg
