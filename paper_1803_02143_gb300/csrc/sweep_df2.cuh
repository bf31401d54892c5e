// sweep_df2.cuh -- forward sweeps of FP64 storage in packed double-float
// arithmetic: every thread carries two independent lanes of work (two
// columns of a strided tile, or two lines of an x1 tile) in float2
// registers and runs the double-float operations as FP32x2 instructions,
// which issue two FP32 operations per instruction on sm_100-class GPUs.
//
// Per lane the arithmetic is that of dfloat.cuh: operands as (hi, lo) float
// pairs, error-free products by FMA, TwoSum into the high word, the rest in
// the low word.  Each 8-byte element is read and written either as an IEEE
// double (split / rebuilt with integer operations) or as a double-float pair
// (IN_DF / OUT_DF), so consecutive sweeps inside a Strang step exchange
// double-float values and convert only at the ends of the step.
#pragma once

#include "sweep_kernels.cuh"

namespace sldg {

__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }

// (sh, sl) = (ah + al)(xh + xl) for two lanes (negations fold into the
// FP32x2 instructions' operands)
__device__ __forceinline__ void df2_first(float2 ah, float2 al, float2 xh, float2 xl, float2& sh,
                                          float2& sl) {
  sh = mul2(ah, xh);
  sl = fma2(ah, xh, neg2(sh));  // error of the product
  sl = fma2(ah, xl, sl);
  sl = fma2(al, xh, sl);
}

// (sh, sl) += (ah + al)(xh + xl) for two lanes, TwoSum on the high word.
__device__ __forceinline__ void df2_mac(float2 ah, float2 al, float2 xh, float2 xl, float2& sh,
                                        float2& sl) {
  const float2 p = mul2(ah, xh);
  const float2 e = fma2(ah, xh, neg2(p));  // p's rounding error
  const float2 t = add2(sh, p);
  const float2 z = add2(t, neg2(sh));
  const float2 err = add2(add2(sh, neg2(add2(t, neg2(z)))), add2(p, neg2(z)));
  sh = t;
  sl = add2(sl, add2(err, e));
  sl = fma2(ah, xl, sl);
  sl = fma2(al, xh, sl);
}

// double -> (hi, lo) with integer operations; |x| < 2^-103 flushes to zero,
// |x| >= 2^128, Inf and NaN become NaN in hi.
__device__ __forceinline__ void dsplit_fast(double x, float& h, float& l) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned fs = __funnelshift_l(lo, hi, 3);  // low 9 exponent bits, 23 mantissa bits
  const unsigned hb = ((fs - 0x40000000u) & 0x7FFFFFFFu) | (hi & 0x80000000u);
  const unsigned cb = (hb & 0xFF800000u) - (23u << 23);
  const unsigned lb = (cb | ((lo >> 6) & 0x7FFFFFu)) + ((lo >> 5) & 1u);
  h = __uint_as_float(hb);
  l = __uint_as_float(lb) - __uint_as_float(cb);
  const unsigned ae = hi & 0x7FF00000u;
  if (ae < (920u << 20)) {
    h = 0.0f;
    l = 0.0f;
  }
  if (ae >= (1151u << 20)) {
    h = __uint_as_float(hb | 0x7FC00000u);
    l = 0.0f;
  }
}

// hi + lo -> double: hi exactly (zero and non-finite kept), lo exactly unless
// it is a float denormal (then off by less than 2^-126), one FP64 add.
__device__ __forceinline__ double djoin_fast(float h, float l) {
  const unsigned uh = __float_as_uint(h), th = uh & 0x7FFFFFFFu;
  unsigned hh = ((th >> 3) + (896u << 20)) | (uh & 0x80000000u);
  unsigned hl = uh << 29;
  if (th < 0x00800000u) {
    hh = uh & 0x80000000u;
    hl = 0u;
  }
  if (th >= 0x7F800000u) hh |= 0x7FF00000u;
  const unsigned ul = __float_as_uint(l), tl = ul & 0x7FFFFFFFu;
  unsigned lh = ((tl >> 3) + (896u << 20)) | (ul & 0x80000000u);
  if (tl == 0u) lh = 0u;
  return __hiloint2double((int)hh, (int)hl) + __hiloint2double((int)lh, (int)(ul << 29));
}

// 8-byte element -> (hi, lo) according to its format
template <bool IN_DF>
__device__ __forceinline__ void load_pair(double raw, float& h, float& l) {
  if (IN_DF) {
    const float2 p = df_unpack(raw);
    h = p.x;
    l = p.y;
  } else {
    dsplit_fast(raw, h, l);
  }
}

template <bool OUT_DF>
__device__ __forceinline__ double store_pair(float h, float l) {
  if (OUT_DF) return df_pack(h, l);
  return djoin_fast(h, l);
}

// One cell of N outputs for two lanes: y = A xa + B xb.  The matrices sit
// in shared memory as float4 (hi lane 0, hi lane 1, lo lane 0, lo lane 1)
// per entry: entries 0..N*N-1 are A (row-major), N*N..2N*N-1 are B.
template <int N, bool OUT_DF>
__device__ __forceinline__ void cell_df2(const float4* __restrict__ M, const float2* xah,
                                         const float2* xal, const float2* xbh, const float2* xbl,
                                         double2* y) {
#pragma unroll
  for (int j = 0; j < N; ++j) {
    float2 sh, sl;
    float4 m = M[j * N];
    df2_first(make_float2(m.x, m.y), make_float2(m.z, m.w), xah[0], xal[0], sh, sl);
#pragma unroll
    for (int l = 1; l < N; ++l) {
      m = M[j * N + l];
      df2_mac(make_float2(m.x, m.y), make_float2(m.z, m.w), xah[l], xal[l], sh, sl);
    }
#pragma unroll
    for (int l = 0; l < N; ++l) {
      m = M[N * N + j * N + l];
      df2_mac(make_float2(m.x, m.y), make_float2(m.z, m.w), xbh[l], xbl[l], sh, sl);
    }
    y[j] = make_double2(store_pair<OUT_DF>(sh.x, sl.x), store_pair<OUT_DF>(sh.y, sl.y));
  }
}

// ---------------------------------------------------------------------------
// Strided forward sweep, FP64 storage, packed double-float.  Requires a
// 16-byte aligned row layout (inner even).  Tile: raw 8-byte elements
// [D][32] staged by cp.async, converted into hi/lo planes [D + N][32] (N zero
// rows at the end stand for source cells outside the zero-inflow box).
// Thread (q, g) owns columns 2q, 2q+1 and cells g, g + 16, ...
// ---------------------------------------------------------------------------
constexpr int kDf2Pairs = kStridedW / 2;                  // 16 column pairs
constexpr int kDf2Groups = kStridedThreads / kDf2Pairs;   // 16 cell groups

inline size_t strided_df2_smem(long long D, int N) {
  return (size_t)D * kStridedW * sizeof(double) + 2 * (size_t)(D + N) * kStridedW * sizeof(float) +
         (size_t)kDf2Pairs * 2 * N * N * sizeof(float4);
}

template <int N, bool PERIODIC, bool PERCOL, bool IN_DF, bool OUT_DF>
__global__ void __launch_bounds__(kStridedThreads, 2)
    k_sweep_strided_df2(double* __restrict__ f, long long inner, int nc, long long ncolblk,
                        const float2* __restrict__ ab2, const int* __restrict__ svec,
                        long long mcount, long long key_div, long long key_mod) {
  constexpr int W = kStridedW, G = kDf2Groups;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int D = nc * N;
  constexpr int MN = 2 * N * N;  // matrix entries per lane pair
  float4* smat = reinterpret_cast<float4*>(smraw);  // [kDf2Pairs][MN], 16-byte aligned first
  double* raw = reinterpret_cast<double*>(smraw + (size_t)kDf2Pairs * MN * sizeof(float4));
  float* th = reinterpret_cast<float*>(raw + (size_t)D * W);
  float* tl = th + (size_t)(D + N) * W;
  const long long cb = blockIdx.x % ncolblk;
  const long long o = blockIdx.x / ncolblk;
  const long long col0 = cb * W;
  const int nvalid = (int)min((long long)W, inner - col0);
  const long long base = o * (long long)D * inner + col0;
  double* fb = f + base;

  // matrices of every lane pair, (hi0, hi1, lo0, lo1) per entry
  for (int e = threadIdx.x; e < kDf2Pairs * MN; e += blockDim.x) {
    const int pq = e / MN, i = e - pq * MN;
    long long k0 = (o / key_div) % key_mod, k1 = k0;
    if (PERCOL) {
      const long long cc = min(col0 + 2 * pq, inner - 1);
      k0 = cc % key_mod;
      k1 = min(cc + 1, inner - 1) % key_mod;
    }
    const float2 a0 = ab2[(long long)i * mcount + k0], a1 = ab2[(long long)i * mcount + k1];
    smat[e] = make_float4(a0.x, a1.x, a0.y, a1.y);
  }
  load_tile_strided<double, true>(raw, fb, inner, D, nvalid);
  const int q = threadIdx.x % kDf2Pairs, g = threadIdx.x / kDf2Pairs;
  const int c0 = 2 * q;
  for (int r = g; r < D; r += G) {
    const double2 v = *reinterpret_cast<const double2*>(raw + r * W + c0);
    float h0, l0, h1, l1;
    load_pair<IN_DF>(v.x, h0, l0);
    load_pair<IN_DF>(v.y, h1, l1);
    *reinterpret_cast<float2*>(th + r * W + c0) = make_float2(h0, h1);
    *reinterpret_cast<float2*>(tl + r * W + c0) = make_float2(l0, l1);
  }
  if (!PERIODIC)
    for (int r = D + g; r < D + N; r += G) {
      *reinterpret_cast<float2*>(th + r * W + c0) = make_float2(0.0f, 0.0f);
      *reinterpret_cast<float2*>(tl + r * W + c0) = make_float2(0.0f, 0.0f);
    }
  __syncthreads();
  if (c0 >= nvalid) return;  // no barrier follows

  const long long k0 = PERCOL ? (col0 + c0) % key_mod : (o / key_div) % key_mod;
  const long long k1 = PERCOL ? (col0 + c0 + 1) % key_mod : k0;
  const float4* M = smat + q * MN;
  int sa0 = -svec[k0] - 1, sa1 = -svec[k1] - 1;
  if (PERIODIC) {
    sa0 = wrap_cell(sa0, nc);
    sa1 = wrap_cell(sa1, nc);
  }
  const bool same = sa0 == sa1;  // both lanes read the same rows: pair loads
  const long long cstride = (long long)N * inner;
  double* out = fb + c0 + (long long)g * cstride;
  for (int c = g; c < nc; c += G, out += G * cstride) {
    int ka0 = c + sa0, ka1 = c + sa1;
    int kb0 = ka0 + 1, kb1 = ka1 + 1;
    if (PERIODIC) {
      if (ka0 >= nc) ka0 -= nc;
      if (kb0 >= nc) kb0 -= nc;
      if (ka1 >= nc) ka1 -= nc;
      if (kb1 >= nc) kb1 -= nc;
    } else {  // out of the box: the zero rows (cell index nc)
      if ((unsigned)ka0 >= (unsigned)nc) ka0 = nc;
      if ((unsigned)kb0 >= (unsigned)nc) kb0 = nc;
      if ((unsigned)ka1 >= (unsigned)nc) ka1 = nc;
      if ((unsigned)kb1 >= (unsigned)nc) kb1 = nc;
    }
    float2 xah[N], xal[N], xbh[N], xbl[N];
    const int ia0 = ka0 * N * W + c0, ia1 = ka1 * N * W + c0 + 1;
    const int ib0 = kb0 * N * W + c0, ib1 = kb1 * N * W + c0 + 1;
    if (same) {
#pragma unroll
      for (int l = 0; l < N; ++l) {
        xah[l] = *reinterpret_cast<const float2*>(th + ia0 + l * W);
        xal[l] = *reinterpret_cast<const float2*>(tl + ia0 + l * W);
        xbh[l] = *reinterpret_cast<const float2*>(th + ib0 + l * W);
        xbl[l] = *reinterpret_cast<const float2*>(tl + ib0 + l * W);
      }
    } else {
#pragma unroll
      for (int l = 0; l < N; ++l) {
        xah[l] = make_float2(th[ia0 + l * W], th[ia1 + l * W]);
        xal[l] = make_float2(tl[ia0 + l * W], tl[ia1 + l * W]);
        xbh[l] = make_float2(th[ib0 + l * W], th[ib1 + l * W]);
        xbl[l] = make_float2(tl[ib0 + l * W], tl[ib1 + l * W]);
      }
    }
    double2 y[N];
    cell_df2<N, OUT_DF>(M, xah, xal, xbh, xbl, y);
#pragma unroll
    for (int j = 0; j < N; ++j) *reinterpret_cast<double2*>(out + (long long)j * inner) = y[j];
  }
}

// ---------------------------------------------------------------------------
// x1 forward sweep, FP64 storage, packed double-float.  A tile is R (even)
// consecutive lines sharing their matrices; lines 2p and 2p+1 form the two
// lanes: planes hold (line 2p, line 2p+1) pairs, [R/2][D] float2 each.  The
// raw staging buffer receives the outputs and is stored contiguously.
// ---------------------------------------------------------------------------
inline size_t x1_df2_smem(long long D, int R, int N) {
  return 2 * (size_t)R * D * sizeof(double) + 2 * (size_t)N * N * sizeof(float4);
}

template <int N, bool IN_DF, bool OUT_DF>
__global__ void __launch_bounds__(kX1Threads, 3)
    k_sweep_x1_df2(double* __restrict__ f, int nc, int R, int tpl_log2,
                   const float2* __restrict__ ab2, const int* __restrict__ svec, long long mcount,
                   long long key_div, long long key_mod) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int D = nc * N;
  const int TL = R * D;
  float4* smat = reinterpret_cast<float4*>(smraw);  // 2N*N entries, broadcast reads
  double* raw = reinterpret_cast<double*>(smraw + 2 * (size_t)N * N * sizeof(float4));
  float2* ph = reinterpret_cast<float2*>(raw + (size_t)TL);
  float2* pl = ph + (size_t)(R / 2) * D;
  double* fb = f + (long long)blockIdx.x * TL;
  const long long key = ((long long)blockIdx.x * R / key_div) % key_mod;
  for (int i = threadIdx.x; i < 2 * N * N; i += blockDim.x) {
    const float2 a = ab2[(long long)i * mcount + key];
    smat[i] = make_float4(a.x, a.x, a.y, a.y);
  }
  for (int i = threadIdx.x; i < TL / 2; i += blockDim.x) cp_async16(raw + 2 * i, fb + 2 * i);
  cp_async_wait_all();
  __syncthreads();
  for (int i = threadIdx.x; i < TL / 2; i += blockDim.x) {
    const int rp = i / D, k = i - rp * D;
    float h0, l0, h1, l1;
    load_pair<IN_DF>(raw[(2 * rp) * D + k], h0, l0);
    load_pair<IN_DF>(raw[(2 * rp + 1) * D + k], h1, l1);
    ph[i] = make_float2(h0, h1);
    pl[i] = make_float2(l0, l1);
  }
  __syncthreads();

  const int sa = wrap_cell(-svec[key] - 1, nc);
  const int TPL = 1 << tpl_log2;
  const int cl = threadIdx.x & (TPL - 1);
  const int rstep = kX1Threads >> tpl_log2;
  for (int rp = threadIdx.x >> tpl_log2; rp < R / 2; rp += rstep) {
    const float2* rh = ph + rp * D;
    const float2* rl = pl + rp * D;
    double* o0 = raw + (2 * rp) * D;
    double* o1 = o0 + D;
    for (int c = cl; c < nc; c += TPL) {
      int ka = c + sa;
      if (ka >= nc) ka -= nc;
      int kb = ka + 1;
      if (kb >= nc) kb -= nc;
      float2 xah[N], xal[N], xbh[N], xbl[N];
#pragma unroll
      for (int l = 0; l < N; ++l) {
        xah[l] = rh[ka * N + l];
        xal[l] = rl[ka * N + l];
        xbh[l] = rh[kb * N + l];
        xbl[l] = rl[kb * N + l];
      }
      double2 y[N];
      cell_df2<N, OUT_DF>(smat, xah, xal, xbh, xbl, y);
#pragma unroll
      for (int j = 0; j < N; ++j) {
        o0[c * N + j] = y[j].x;  // raw is fully converted and no longer read
        o1[c * N + j] = y[j].y;
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < TL / 2; i += blockDim.x)
    reinterpret_cast<double2*>(fb)[i] = reinterpret_cast<const double2*>(raw)[i];
}

template <int N, bool IN_DF, bool OUT_DF>
cudaError_t launch_strided_df3_T(const SweepArgs& a, cudaStream_t st);
template <int N, bool IN_DF, bool OUT_DF>
cudaError_t launch_x1_df3_T(const SweepArgs& a, cudaStream_t st);
template <int N, bool IN_DF, bool OUT_DF>
cudaError_t launch_x1_warp_T(const SweepArgs& a, cudaStream_t st);

// Launch the packed kernels when they apply (forward, degree <= 2, aligned
// layout, even x1 tile height); returns cudaErrorNotSupported otherwise.
template <int N, bool IN_DF, bool OUT_DF>
cudaError_t launch_sweep_df2_T(const SweepArgs& a, cudaStream_t st) {
  double* f = reinterpret_cast<double*>(a.f);
  const float2* ab2 = reinterpret_cast<const float2*>(a.ab2);
  const long long D = (long long)a.nc * N;
  if (a.adjoint || (reinterpret_cast<uintptr_t>(f) & 15)) return cudaErrorNotSupported;
  if (a.dim == 0) {
    if (out_of_place(a)) return cudaErrorNotSupported;
    {
      cudaError_t e3 = launch_x1_warp_T<N, IN_DF, OUT_DF>(a, st);
      if (e3 != cudaErrorNotSupported) return e3;
      e3 = launch_x1_df3_T<N, IN_DF, OUT_DF>(a, st);
      if (e3 != cudaErrorNotSupported) return e3;
    }
    const int R = a.lines_per_tile;
    if (R % 2) return cudaErrorNotSupported;
    const size_t smem = x1_df2_smem(D, R, N);
    auto kfn = k_sweep_x1_df2<N, IN_DF, OUT_DF>;
    cudaError_t e = set_smem(kfn, smem);
    if (e != cudaSuccess) return e;
    kfn<<<(unsigned)(a.outer / R), kX1Threads, smem, st>>>(f, a.nc, R, x1_tpl_log2(a.nc), ab2, a.s,
                                                           a.mcount, a.key_div, a.key_mod);
    return cudaGetLastError();
  }
  if (a.inner % 2) return cudaErrorNotSupported;
  {
    const cudaError_t e3 = launch_strided_df3_T<N, IN_DF, OUT_DF>(a, st);
    if (e3 != cudaErrorNotSupported || out_of_place(a)) return e3;
  }
  const size_t smem = strided_df2_smem(D, N);
  if (smem > 227 * 1024) return cudaErrorNotSupported;
  const long long ncolblk = (a.inner + kStridedW - 1) / kStridedW;
  const long long blocks = ncolblk * a.outer;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  auto kfn = a.dim < 2 ? k_sweep_strided_df2<N, true, false, IN_DF, OUT_DF>
                       : (a.periodic ? k_sweep_strided_df2<N, true, true, IN_DF, OUT_DF>
                                     : k_sweep_strided_df2<N, false, true, IN_DF, OUT_DF>);
  cudaError_t e = set_smem(kfn, smem);
  if (e != cudaSuccess) return e;
  kfn<<<(unsigned)blocks, kStridedThreads, smem, st>>>(f, a.inner, a.nc, ncolblk, ab2, a.s,
                                                       a.mcount, a.key_div, a.key_mod);
  return cudaGetLastError();
}

template <int N>
cudaError_t launch_sweep_df2_N(const SweepArgs& a, cudaStream_t st) {
  if (a.in_df && a.out_df) return launch_sweep_df2_T<N, true, true>(a, st);
  if (a.in_df) return launch_sweep_df2_T<N, true, false>(a, st);
  if (a.out_df) return launch_sweep_df2_T<N, false, true>(a, st);
  return launch_sweep_df2_T<N, false, false>(a, st);
}

inline cudaError_t launch_sweep_df2(const SweepArgs& a, cudaStream_t st) {
  switch (a.n) {
    case 1: return launch_sweep_df2_N<1>(a, st);
    case 2: return launch_sweep_df2_N<2>(a, st);
    case 3: return launch_sweep_df2_N<3>(a, st);
    default: return cudaErrorNotSupported;
  }
}

}  // namespace sldg
