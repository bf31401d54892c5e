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
// Each CTA stages whole lines in shared memory (cp.async, all bytes of the
// tile in flight at once) before writing any output, so the update is in
// place: every line is owned by exactly one CTA and is read completely before
// the first store to it.
//
// Arithmetic policies:
//   PolF32  float storage, FP32 FMA;
//   PolF64  double storage, FP64 FMA (the FP64 pipe of GB300 does about two
//           FMA per clock per SM, so this path is bound by it);
//   PolDF   double storage, double-float arithmetic on the FP32 pipe: each
//           double is split into a (hi, lo) float pair with integer bit
//           operations, products are made error-free with FMA and summed with
//           TwoSum (Knuth), and the result is rebuilt as a double with integer
//           operations and one FP64 add.  About 2^-47 relative accuracy.
#pragma once

#include <type_traits>

#include "ctx.h"
#include "dfloat.cuh"

namespace sldg {

constexpr int kStridedW = 32;  // columns per tile of a strided sweep
constexpr int kStridedThreads = 256;
constexpr int kStridedGroups = kStridedThreads / kStridedW;
constexpr int kX1Threads = 256;

// ---------------------------------------------------------------------------
// cp.async helpers (global -> shared without a register round trip)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async8(void* sdst, const void* gsrc) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async4(void* sdst, const void* gsrc) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

template <int BYTES>
__device__ __forceinline__ void cp_async_elem(void* sdst, const void* gsrc) {
  if (BYTES == 8) cp_async8(sdst, gsrc);
  else cp_async4(sdst, gsrc);
}

// ---------------------------------------------------------------------------
// Policies: storage type S, shared tile element E, matrix element M.
// ---------------------------------------------------------------------------
struct PolF32 {
  using S = float;
  using E = float;
  using M = float;
  static constexpr bool kSplit = false;
  __device__ static E conv(S x) { return x; }
};
struct PolF64 {
  using S = double;
  using E = double;
  using M = double;
  static constexpr bool kSplit = false;
  __device__ static E conv(S x) { return x; }
};
// IN_DF / OUT_DF: the 8-byte elements are read / written as double-float
// pairs instead of IEEE doubles (sub-steps inside a Strang step).
template <bool IN_DF, bool OUT_DF>
struct PolDFT {
  using S = double;
  using E = float2;
  using M = float2;
  static constexpr bool kSplit = true;
  __device__ static E conv(S x) { return IN_DF ? df_unpack(x) : dsplit(x); }
  __device__ static S store(float h, float l) { return OUT_DF ? df_pack(h, l) : djoin(h, l); }
};
using PolDF = PolDFT<false, false>;

// y[j] = sum_l M1[j,l] xa[l] + M2[j,l] xb[l] (or the transposes) for one cell.
template <class P, int N, bool ADJ>
__device__ __forceinline__ void cell_apply(const typename P::M* A, const typename P::M* B,
                                           const typename P::E* xa, const typename P::E* xb,
                                           typename P::S* y) {
  if constexpr (P::kSplit) {
#pragma unroll
    for (int j = 0; j < N; ++j) {
      float sh, sl;
      const float2 a0 = ADJ ? A[j] : A[j * N];
      df_first(a0.x, a0.y, xa[0], sh, sl);
#pragma unroll
      for (int l = 1; l < N; ++l) {
        const float2 a = ADJ ? A[l * N + j] : A[j * N + l];
        df_mac(a.x, a.y, xa[l], sh, sl);
      }
#pragma unroll
      for (int l = 0; l < N; ++l) {
        const float2 b = ADJ ? B[l * N + j] : B[j * N + l];
        df_mac(b.x, b.y, xb[l], sh, sl);
      }
      y[j] = P::store(sh, sl);
    }
  } else {
#pragma unroll
    for (int j = 0; j < N; ++j) {
      typename P::S acc = 0;
#pragma unroll
      for (int l = 0; l < N; ++l) {
        acc = fma(ADJ ? A[l * N + j] : A[j * N + l], xa[l], acc);
        acc = fma(ADJ ? B[l * N + j] : B[j * N + l], xb[l], acc);
      }
      y[j] = acc;
    }
  }
}

template <class P>
__device__ __forceinline__ typename P::E zero_elem() {
  if constexpr (P::kSplit) return make_float2(0.0f, 0.0f);
  else return typename P::E(0);
}

// ---------------------------------------------------------------------------
// Tile load: rows r < D of the kStridedW columns starting at gsrc (row stride
// `inner` elements) into tile[r][col] (raw storage elements).  VEC: every row
// segment is 16-byte aligned and the valid width is a multiple of 16 bytes.
// ---------------------------------------------------------------------------
template <typename S, bool VEC>
__device__ __forceinline__ void load_tile_strided(S* tile, const S* gsrc, long long inner, int D,
                                                  int ncols_valid) {
  constexpr int W = kStridedW;
  if (VEC) {
    constexpr int PER = 16 / sizeof(S);          // elements per chunk
    constexpr int CPR = W / PER;                 // chunks per full row
    const int vchunks = ncols_valid / PER;       // valid chunks per row
    const int total = D * CPR;
    for (int i = threadIdx.x; i < total; i += blockDim.x) {
      const int r = i / CPR, q = i - r * CPR;
      if (q < vchunks) cp_async16(tile + r * W + q * PER, gsrc + (long long)r * inner + q * PER);
    }
  } else {
    const int lane = threadIdx.x & (W - 1), grp = threadIdx.x / W;
    if (lane < ncols_valid)
      for (int r = grp; r < D; r += kStridedGroups)
        cp_async_elem<sizeof(S)>(tile + r * W + lane, gsrc + (long long)r * inner + lane);
  }
  cp_async_wait_all();
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Strided sweep (x2, v1, v2): f viewed as [outer][D][inner]; a tile is one
// outer index and kStridedW consecutive inner columns, all D rows.
//   PERCOL: matrix key per column (v-sweeps: key = column % key_mod, the
//           x-node); else per tile (x2-sweep: key = (outer / key_div) % key_mod).
//   EBAR:   also accumulate d/dE <out_bar, S(E) g> per column into epart
//           (adjoint v-sweeps, PolF32/PolF64 only); g is the forward input.
// ---------------------------------------------------------------------------
template <class P, int N, bool PERIODIC, bool PERCOL, bool ADJ, bool EBAR, bool VEC>
__global__ void __launch_bounds__(kStridedThreads)
    k_sweep_strided(typename P::S* __restrict__ f, const typename P::S* __restrict__ gfwd,
                    double* __restrict__ epart, long long inner, int nc, long long ncolblk,
                    const typename P::M* __restrict__ ab, const typename P::S* __restrict__ dab,
                    const int* __restrict__ svec, long long mcount, long long key_div,
                    long long key_mod) {
  using S = typename P::S;
  using E = typename P::E;
  using M = typename P::M;
  constexpr int W = kStridedW, G = kStridedGroups;
  extern __shared__ __align__(16) unsigned char smraw[];
  S* rawtile = reinterpret_cast<S*>(smraw);
  E* tile = reinterpret_cast<E*>(smraw);  // same footprint: sizeof(E) == sizeof(S)
  const int D = nc * N;
  const long long cb = blockIdx.x % ncolblk;
  const long long o = blockIdx.x / ncolblk;
  const int lane = threadIdx.x & (W - 1);
  const int grp = threadIdx.x / W;
  const long long col0 = cb * W;
  const long long col = col0 + lane;
  const int nvalid = (int)min((long long)W, inner - col0);
  const bool valid = lane < nvalid;
  const long long base = o * (long long)D * inner + col0;
  S* fb = f + base;

  load_tile_strided<S, VEC>(rawtile, fb, inner, D, nvalid);
  if constexpr (P::kSplit) {
    // convert in place, each thread its own elements (no cross-thread hazard)
    if (valid)
      for (int r = grp; r < D; r += G) tile[r * W + lane] = P::conv(rawtile[r * W + lane]);
    __syncthreads();
  }

  double eacc = 0.0;
  if (valid) {
    const long long key = PERCOL ? (col % key_mod) : ((o / key_div) % key_mod);
    M A[N * N], B[N * N];
#pragma unroll
    for (int i = 0; i < N * N; ++i) {
      A[i] = ab[(long long)i * mcount + key];
      B[i] = ab[(long long)(N * N + i) * mcount + key];
    }
    const int s = svec[key];
    // source cells of target c: c + sa (A) and c + sa + 1 (B) forward,
    // c + sa and c + sa - 1 transposed
    int sa = ADJ ? s + 1 : -s - 1;
    if (PERIODIC) sa = wrap_cell(sa, nc);
    const long long cstride = (long long)N * inner;
    S* out = fb + lane + (long long)grp * cstride;
    for (int c = grp; c < nc; c += G, out += G * cstride) {
      int ka = c + sa;
      int kb = ADJ ? ka - 1 : ka + 1;
      bool va = true, vb = true;
      if (PERIODIC) {
        if (ka >= nc) ka -= nc;
        if (kb >= nc) kb -= nc;
        if (kb < 0) kb += nc;
      } else {
        va = (unsigned)ka < (unsigned)nc;
        vb = (unsigned)kb < (unsigned)nc;
      }
      E xa[N], xb[N];
      const E* ra = tile + ka * N * W + lane;
      const E* rb = tile + kb * N * W + lane;
#pragma unroll
      for (int l = 0; l < N; ++l) {
        xa[l] = va ? ra[l * W] : zero_elem<P>();
        xb[l] = vb ? rb[l * W] : zero_elem<P>();
      }
      S y[N];
      cell_apply<P, N, ADJ>(A, B, xa, xb, y);
#pragma unroll
      for (int j = 0; j < N; ++j) out[(long long)j * inner] = y[j];
    }
    if constexpr (EBAR && !P::kSplit) {
      // d/dtheta of <lam_out, S g>: lam_out[c] is the staged tile, g at the
      // forward source cells c-s-1, c-s.
      S dA[N * N], dB[N * N];
#pragma unroll
      for (int i = 0; i < N * N; ++i) {
        dA[i] = dab[(long long)i * mcount + key];
        dB[i] = dab[(long long)(N * N + i) * mcount + key];
      }
      const S* gb = gfwd + base;
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
        S ga[N], gbv[N];
#pragma unroll
        for (int l = 0; l < N; ++l) {
          ga[l] = va ? gb[(long long)(ka * N + l) * inner + lane] : S(0);
          gbv[l] = vb ? gb[(long long)(kb * N + l) * inner + lane] : S(0);
        }
        S cell = S(0);
#pragma unroll
        for (int j = 0; j < N; ++j) {
          S d = S(0);
#pragma unroll
          for (int l = 0; l < N; ++l) {
            d = fma(dA[j * N + l], ga[l], d);
            d = fma(dB[j * N + l], gbv[l], d);
          }
          cell = fma(rawtile[(c * N + j) * W + lane], d, cell);
        }
        eacc += (double)cell;
      }
    }
  }
  if constexpr (EBAR) {
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
// D1, so all lines of a tile share their v1 node and matrices).  The tile is
// staged with 16-byte cp.async (or element-wise when the line is not a
// multiple of 16 bytes), outputs are staged and stored contiguously.
// Threads cover TPL cells of a line (TPL a power of two >= the cell count
// when it fits, else 256) and 256/TPL lines per pass.
// ---------------------------------------------------------------------------
template <class P, int N, bool ADJ, bool VEC>
__global__ void __launch_bounds__(kX1Threads)
    k_sweep_x1(typename P::S* __restrict__ f, int nc, int R, int tpl_log2,
               const typename P::M* __restrict__ ab, const int* __restrict__ svec,
               long long mcount, long long key_div, long long key_mod) {
  using S = typename P::S;
  using E = typename P::E;
  using M = typename P::M;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int D = nc * N;
  const int TL = R * D;
  const int TLp = (TL + 1) & ~1;  // keep the output buffer 16-byte aligned
  S* rin = reinterpret_cast<S*>(smraw);
  E* sin = reinterpret_cast<E*>(smraw);
  S* sout = rin + (sizeof(S) == 8 ? TLp : ((TL + 3) & ~3));
  const long long t0 = (long long)blockIdx.x * TL;
  S* fb = f + t0;
  constexpr int V = 16 / sizeof(S);
  if (VEC) {
    for (int i = threadIdx.x; i < TL / V; i += blockDim.x) cp_async16(rin + i * V, fb + i * V);
  } else {
    for (int i = threadIdx.x; i < TL; i += blockDim.x) cp_async_elem<sizeof(S)>(rin + i, fb + i);
  }
  cp_async_wait_all();
  __syncthreads();
  if constexpr (P::kSplit) {
    for (int i = threadIdx.x; i < TL; i += blockDim.x) sin[i] = P::conv(rin[i]);
    __syncthreads();
  }

  const long long L0 = (long long)blockIdx.x * R;
  const long long key = (L0 / key_div) % key_mod;
  M A[N * N], B[N * N];
#pragma unroll
  for (int i = 0; i < N * N; ++i) {
    A[i] = ab[(long long)i * mcount + key];
    B[i] = ab[(long long)(N * N + i) * mcount + key];
  }
  const int s = svec[key];
  int sa = wrap_cell(ADJ ? s + 1 : -s - 1, nc);
  const int TPL = 1 << tpl_log2;
  const int cl = threadIdx.x & (TPL - 1);
  const int r0 = threadIdx.x >> tpl_log2;
  const int rstep = kX1Threads >> tpl_log2;
  for (int r = r0; r < R; r += rstep) {
    const E* row = sin + r * D;
    S* orow = sout + r * D;
    for (int c = cl; c < nc; c += TPL) {
      int ka = c + sa;
      if (ka >= nc) ka -= nc;
      int kb = ADJ ? ka - 1 : ka + 1;
      if (kb >= nc) kb -= nc;
      if (kb < 0) kb += nc;
      E xa[N], xb[N];
#pragma unroll
      for (int l = 0; l < N; ++l) {
        xa[l] = row[ka * N + l];
        xb[l] = row[kb * N + l];
      }
      S y[N];
      cell_apply<P, N, ADJ>(A, B, xa, xb, y);
#pragma unroll
      for (int j = 0; j < N; ++j) orow[c * N + j] = y[j];
    }
  }
  __syncthreads();
  if (VEC) {
    using V4 = typename std::conditional<sizeof(S) == 8, double2, float4>::type;
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
  size_t TLp = esize == 8 ? ((TL + 1) & ~(size_t)1) : ((TL + 3) & ~(size_t)3);
  return (TLp + TL) * esize;
}

inline int x1_tpl_log2(int nc) {
  int l = 0;
  while ((1 << l) < nc && l < 8) ++l;
  return l;
}

// Opt in to more than 48 KB of dynamic shared memory and ask for the
// largest shared-memory carveout, so several large tiles fit on one SM.
template <class KF>
cudaError_t set_smem(KF kfn, size_t smem) {
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  if (smem > 16 * 1024)
    return cudaFuncSetAttribute(kfn, cudaFuncAttributePreferredSharedMemoryCarveout,
                                (int)cudaSharedmemCarveoutMaxShared);
  return cudaSuccess;
}

template <class P, int N>
cudaError_t launch_sweep_T(const SweepArgs& a, cudaStream_t st) {
  using S = typename P::S;
  using M = typename P::M;
  S* f = reinterpret_cast<S*>(a.f);
  const M* ab = reinterpret_cast<const M*>(P::kSplit ? a.ab2 : a.ab);
  const S* dab = reinterpret_cast<const S*>(a.dab);
  const long long D = (long long)a.nc * N;
  if (a.dim == 0) {
    const int R = a.lines_per_tile;
    const long long tiles = a.outer / R;  // for x1, outer = number of lines
    const size_t smem = x1_smem(sizeof(S), D, R);
    const bool vec = ((long long)R * D * sizeof(S)) % 16 == 0 && (reinterpret_cast<uintptr_t>(f) & 15) == 0;
    auto kfn = a.adjoint ? (vec ? k_sweep_x1<P, N, true, true> : k_sweep_x1<P, N, true, false>)
                         : (vec ? k_sweep_x1<P, N, false, true> : k_sweep_x1<P, N, false, false>);
    cudaError_t e = set_smem(kfn, smem);
    if (e != cudaSuccess) return e;
    kfn<<<(unsigned)tiles, kX1Threads, smem, st>>>(f, a.nc, R, x1_tpl_log2(a.nc), ab, a.s, a.mcount,
                                                   a.key_div, a.key_mod);
    return cudaGetLastError();
  }
  const long long ncolblk = (a.inner + kStridedW - 1) / kStridedW;
  const long long blocks = ncolblk * a.outer;
  const size_t smem = strided_smem(sizeof(S), D);
  const S* g = reinterpret_cast<const S*>(a.g);
  const bool vec = (a.inner * (long long)sizeof(S)) % 16 == 0 && (reinterpret_cast<uintptr_t>(f) & 15) == 0;
  const bool percol = a.dim >= 2;
  const bool ebar = a.adjoint && percol && a.g != nullptr && a.epart != nullptr;
  using KFn = decltype(&k_sweep_strided<P, N, true, false, false, false, true>);
  KFn kfn;
#define SLDG_PICK(PER, PC, ADJ, EB)                                                      \
  kfn = vec ? k_sweep_strided<P, N, PER, PC, ADJ, EB, true>                              \
            : k_sweep_strided<P, N, PER, PC, ADJ, EB, false>
  if (!percol) {
    if (a.adjoint) SLDG_PICK(true, false, true, false);
    else SLDG_PICK(true, false, false, false);
  } else if (a.periodic) {
    if (!a.adjoint) SLDG_PICK(true, true, false, false);
    else if (ebar) SLDG_PICK(true, true, true, true);
    else SLDG_PICK(true, true, true, false);
  } else {
    if (!a.adjoint) SLDG_PICK(false, true, false, false);
    else if (ebar) SLDG_PICK(false, true, true, true);
    else SLDG_PICK(false, true, true, false);
  }
#undef SLDG_PICK
  cudaError_t e = set_smem(kfn, smem);
  if (e != cudaSuccess) return e;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  kfn<<<(unsigned)blocks, kStridedThreads, smem, st>>>(f, g, a.epart, a.inner, a.nc, ncolblk, ab,
                                                       dab, a.s, a.mcount, a.key_div, a.key_mod);
  return cudaGetLastError();
}

template <class P>
cudaError_t launch_sweep_any(const SweepArgs& a, cudaStream_t st) {
  switch (a.n) {
    case 1: return launch_sweep_T<P, 1>(a, st);
    case 2: return launch_sweep_T<P, 2>(a, st);
    case 3: return launch_sweep_T<P, 3>(a, st);
    case 4: return launch_sweep_T<P, 4>(a, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace sldg
