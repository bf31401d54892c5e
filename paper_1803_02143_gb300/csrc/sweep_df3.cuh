// sweep_df3.cuh -- strided forward sweeps (x2, v1, v2) of FP64 storage in
// packed double-float arithmetic, organised to keep the instruction count
// per nodal value low:
//   - a CTA owns a column block of 32 columns and walks several outer
//     indices (tiles) with it, so the per-column matrices of the v-sweeps
//     are staged once per CTA;
//   - thread (q, g) owns the column pair 2q, 2q+1 (the two lanes of every
//     FP32x2 instruction) and a run of consecutive cells, so each source
//     cell is read from shared memory and converted once (the b-cell of
//     output c is the a-cell of output c+1);
//   - the staged tile keeps the raw 8-byte elements; there is no separate
//     conversion pass, and outputs go straight to global memory as double2.
// All index arithmetic inside a tile is 32-bit.
#pragma once

#include "sweep_df2.cuh"

namespace sldg {

constexpr int kDf3Threads = 256;
constexpr int kDf3Pairs = kStridedW / 2;             // 16 column pairs
constexpr int kDf3Groups = kDf3Threads / kDf3Pairs;  // 16 cell runs
constexpr int kDf3TilesPerCtaV = 8;  // outer indices walked by one CTA: v-sweeps
constexpr int kDf3TilesPerCtaX = 8;  // x2 sweep

// float4 entries per lane pair: odd, so the 16 pairs' matrix reads of a
// quarter warp fall in distinct banks
template <int N>
__host__ __device__ constexpr int df3_mat_stride() {
  return 2 * N * N + 1;
}

// matrices, then nbuf tile buffers of D + N rows (N zero rows each)
template <int N, bool PERCOL>
inline size_t strided_df3_smem(long long D, int nbuf) {
  const size_t mats = PERCOL ? (size_t)kDf3Pairs * df3_mat_stride<N>() : (size_t)(2 * N * N);
  return mats * sizeof(float4) + nbuf * (size_t)(D + N) * kStridedW * sizeof(double);
}

// Tile conversion in place: each 16-byte column pair of a staged row,
// (x_c0, x_c0+1) as IEEE doubles or packed double-float elements, becomes
// (h_c0, h_c0+1, l_c0, l_c0+1), so that lane-packed operands load directly
// into register pairs.
template <bool IN_DF>
__device__ __forceinline__ void df3_pair_planar(double* __restrict__ raw, int chunks) {
  for (int i = threadIdx.x; i < chunks; i += blockDim.x) {
    float4* p = reinterpret_cast<float4*>(raw) + i;
    const double2 v = *reinterpret_cast<const double2*>(p);
    float h0, l0, h1, l1;
    load_pair<IN_DF>(v.x, h0, l0);
    load_pair<IN_DF>(v.y, h1, l1);
    *p = make_float4(h0, h1, l0, l1);
  }
}

// Source cell of both lanes from a pair-planar tile.  SAME: both lanes read
// cell k0 (one 16-byte load per node).  Else lane 0 reads cell k0 and lane 1
// cell k1 (per-column shifts that differ across the pair).
template <int N, bool SAME>
__device__ __forceinline__ void df3_load_cell(const double* __restrict__ raw, int c0, int k0, int k1,
                                              float2* xh, float2* xl) {
  constexpr int W = kStridedW;
#pragma unroll
  for (int l = 0; l < N; ++l) {
    const float4 u0 = *reinterpret_cast<const float4*>(raw + (k0 * N + l) * W + c0);
    if (SAME) {
      xh[l] = make_float2(u0.x, u0.y);
      xl[l] = make_float2(u0.z, u0.w);
    } else {
      const float4 u1 = *reinterpret_cast<const float4*>(raw + (k1 * N + l) * W + c0);
      xh[l] = make_float2(u0.x, u1.y);
      xl[l] = make_float2(u0.z, u1.w);
    }
  }
}

// y = A xa + B xb for one cell of both lanes: the 2N source terms in order
// (A columns, then B columns), each applied to all N outputs, so the N
// double-float accumulations are independent chains.  An empty asm with a
// memory clobber per term keeps that term's matrix reads next to their use
// (loading all 2N^2 float4 entries of a cell up front would spill).
template <int N>
__device__ __forceinline__ void df3_accumulate(const float4* __restrict__ M, const float2* ah,
                                               const float2* al, const float2* bh,
                                               const float2* bl, float2* sh, float2* sl) {
#pragma unroll
  for (int t = 0; t < 2 * N; ++t) {
    asm volatile("" ::: "memory");
    const float2 xh = t < N ? ah[t] : bh[t - N];
    const float2 xl = t < N ? al[t] : bl[t - N];
#pragma unroll
    for (int j = 0; j < N; ++j) {
      const float4 m = M[t < N ? j * N + t : N * N + j * N + (t - N)];
      if (t == 0) df2_first(make_float2(m.x, m.y), make_float2(m.z, m.w), xh, xl, sh[j], sl[j]);
      else df2_mac(make_float2(m.x, m.y), make_float2(m.z, m.w), xh, xl, sh[j], sl[j]);
    }
  }
}

// The same for the R outputs j0 .. j0 + R - 1 of a cell only.
template <int N, int R>
__device__ __forceinline__ void df3_accumulate_rows(const float4* __restrict__ M, int j0,
                                                    const float2* ah, const float2* al,
                                                    const float2* bh, const float2* bl,
                                                    float2* sh, float2* sl) {
#pragma unroll
  for (int t = 0; t < 2 * N; ++t) {
    asm volatile("" ::: "memory");
    const float2 xh = t < N ? ah[t] : bh[t - N];
    const float2 xl = t < N ? al[t] : bl[t - N];
#pragma unroll
    for (int jj = 0; jj < R; ++jj) {
      const int j = j0 + jj;
      const float4 m = M[t < N ? j * N + t : N * N + j * N + (t - N)];
      if (t == 0) df2_first(make_float2(m.x, m.y), make_float2(m.z, m.w), xh, xl, sh[jj], sl[jj]);
      else df2_mac(make_float2(m.x, m.y), make_float2(m.z, m.w), xh, xl, sh[jj], sl[jj]);
    }
  }
}

template <int N, bool OUT_DF>
__device__ __forceinline__ void df3_cell(const float4* __restrict__ M, const float2* ah,
                                         const float2* al, const float2* bh, const float2* bl,
                                         double* out, long long rstride) {
  float2 sh[N], sl[N];
  df3_accumulate<N>(M, ah, al, bh, bl, sh, sl);
#pragma unroll
  for (int j = 0; j < N; ++j)
    *reinterpret_cast<double2*>(out + j * rstride) =
        make_double2(store_pair<OUT_DF>(sh[j].x, sl[j].x), store_pair<OUT_DF>(sh[j].y, sl[j].y));
}

// Outputs cb .. ce-1 of one column pair: a sliding window over the source
// cells (the b-cell of output c is the a-cell of output c + 1).  Source cells
// step along the line with a periodic wrap, or map to the zero cell nc
// outside a zero-inflow box.
template <int N, bool PERIODIC, bool SAME, bool OUT_DF>
__device__ __forceinline__ void df3_run(const double* __restrict__ raw, const float4* __restrict__ M,
                                        int c0, int cb, int ce, int sa0, int sa1, int nc,
                                        double* fb, long long rstride) {
  int k0 = cb + sa0, k1 = cb + sa1;
  if (PERIODIC) {
    if (k0 >= nc) k0 -= nc;
    if (k1 >= nc) k1 -= nc;
  }
  auto next = [nc](int k) {
    if (PERIODIC) return k + 1 == nc ? 0 : k + 1;
    return k + 1;
  };
  auto row = [nc](int k) {
    if (PERIODIC) return k;
    return (unsigned)k < (unsigned)nc ? k : nc;
  };
  float2 uh[N], ul[N], wh[N], wl[N];
  df3_load_cell<N, SAME>(raw, c0, row(k0), row(k1), uh, ul);
  double* out = fb + c0 + (long long)cb * N * rstride;
  const long long cstep = (long long)N * rstride;
  int c = cb;
  if constexpr (N <= 3) {
    // two cells per iteration, the two register sets trading the a and b
    // roles (no window copies; 4% faster v-sweeps at 192-node v-lines, and
    // slower at four nodes per cell, where the registers run out)
#pragma unroll 1
    for (; c + 1 < ce; c += 2, out += 2 * cstep) {
      k0 = next(k0);
      k1 = next(k1);
      df3_load_cell<N, SAME>(raw, c0, row(k0), row(k1), wh, wl);
      df3_cell<N, OUT_DF>(M, uh, ul, wh, wl, out, rstride);
      k0 = next(k0);
      k1 = next(k1);
      df3_load_cell<N, SAME>(raw, c0, row(k0), row(k1), uh, ul);
      df3_cell<N, OUT_DF>(M, wh, wl, uh, ul, out + cstep, rstride);
    }
  }
#pragma unroll 1
  for (; c < ce; ++c, out += cstep) {
    k0 = next(k0);
    k1 = next(k1);
    df3_load_cell<N, SAME>(raw, c0, row(k0), row(k1), wh, wl);
    df3_cell<N, OUT_DF>(M, uh, ul, wh, wl, out, rstride);
#pragma unroll
    for (int l = 0; l < N; ++l) {
      uh[l] = wh[l];
      ul[l] = wl[l];
    }
  }
}

// A tile is 32 of the ncols columns of one outer index o, all D rows:
// element (o, row r, column c) sits at o * ostride + r * rstride + c.
// PERCOL (v-sweeps): matrix and shift per column (key = column, the
// x-node), periodic or zero inflow; consecutive outer indices of a CTA share
// its matrices.  Else (x2-sweep, periodic): one matrix per tile, key =
// (o / key_div) % key_mod.
// With two tile buffers (nbuf = 2) the next tile is loaded (cp.async) while
// the current one is computed; two CTAs per SM (105 KB of shared memory per
// CTA for 192-node lines).  Longer lines use one buffer.
template <int N, bool PERIODIC, bool PERCOL, bool IN_DF, bool OUT_DF>
__global__ void __launch_bounds__(kDf3Threads, N <= 2 ? 3 : 2)
    k_sweep_strided_df3(const double* f, double* out, int ncols, long long rstride, long long ostride,
                        int nc, int outer, int nbuf, const float2* __restrict__ ab2,
                        const int* __restrict__ svec, long long mcount, int key_div, int key_mod) {
  static_assert(PERCOL || PERIODIC, "the per-tile matrix form serves the periodic x2 sweep");
  constexpr int W = kStridedW;
  constexpr int MN = 2 * N * N;
  constexpr int MS = PERCOL ? df3_mat_stride<N>() : MN;
  extern __shared__ __align__(16) unsigned char smraw[];
  float4* smat = reinterpret_cast<float4*>(smraw);
  double* raw =
      reinterpret_cast<double*>(smraw + (size_t)(PERCOL ? kDf3Pairs * MS : MN) * sizeof(float4));
  const int D = nc * N;
  const int col0 = blockIdx.x * W;
  const int nvalid = min(W, ncols - col0);
  const int q = threadIdx.x % kDf3Pairs, g = threadIdx.x / kDf3Pairs;
  const int c0 = 2 * q;
  const int cb = (g * nc) / kDf3Groups, ce = ((g + 1) * nc) / kDf3Groups;
  const bool active = c0 < nvalid && cb < ce;

  // a-cell offset per lane: the source a-cell of output c is c + sa
  // (periodic: sa in [0, nc) and the sum taken mod nc)
  int sa0 = 0, sa1 = 0;
  if (PERCOL) {
    for (int e = threadIdx.x; e < kDf3Pairs * MN; e += blockDim.x) {
      const int pq = e / MN, i = e - pq * MN;
      const int k0 = min(col0 + 2 * pq, ncols - 1), k1 = min(col0 + 2 * pq + 1, ncols - 1);
      const float2 a0 = ab2[(long long)i * mcount + k0], a1 = ab2[(long long)i * mcount + k1];
      smat[pq * MS + i] = make_float4(a0.x, a1.x, a0.y, a1.y);
    }
    sa0 = -svec[min(col0 + c0, ncols - 1)] - 1;
    sa1 = -svec[min(col0 + c0 + 1, ncols - 1)] - 1;
    if (PERIODIC) {
      sa0 = wrap_cell(sa0, nc);
      sa1 = wrap_cell(sa1, nc);
    }
  }
  const int bstride = (D + N) * W;  // doubles per tile buffer
  if (!PERIODIC)  // the zero cell, rows D .. D+N-1 of each buffer (never loaded)
    for (int i = threadIdx.x; i < N * W; i += blockDim.x) {
      raw[D * W + i] = 0.0;
      if (nbuf == 2) raw[bstride + D * W + i] = 0.0;
    }
  const float4* M = PERCOL ? smat + q * MS : smat;
  const int chunks = D * (W / 2);  // 16-byte chunks of a full tile
  const int vchunks = nvalid / 2;  // valid chunks per row

  auto issue = [&](int o, double* dst) {
    const double* src = f + (long long)o * ostride + col0;
    for (int i = threadIdx.x; i < chunks; i += blockDim.x) {
      const int r = i / (W / 2), cq = i - r * (W / 2);
      if (cq < vchunks) cp_async16(dst + r * W + 2 * cq, src + r * rstride + 2 * cq);
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
  // outer indices of this CTA: o0, o0 + ostep, ... below o1.  v-sweeps stride
  // by the grid (their matrices are per column); the x2 sweep takes a
  // contiguous run so that its per-tile matrix (one v2 node per D2
  // consecutive planes) is restaged only when the node changes.
  int o0, o1, ostep;
  if (PERCOL) {
    o0 = blockIdx.y;
    o1 = outer;
    ostep = gridDim.y;
  } else {
    const int per = (outer + gridDim.y - 1) / gridDim.y;
    o0 = blockIdx.y * per;
    o1 = min(outer, o0 + per);
    ostep = 1;
  }
  int key_cur = -1;
  if (nbuf == 2 && o0 < o1) issue(o0, raw);
  int b = 0;
  for (int o = o0; o < o1; o += ostep, b ^= 1) {
    double* fb = out + (long long)o * ostride + col0;
    double* cur = raw + (nbuf == 2 ? b : 0) * bstride;
    if (nbuf == 1) issue(o, cur);
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    if (!PERCOL) {
      const int key = (o / key_div) % key_mod;
      if (key != key_cur) {  // uniform over the CTA
        for (int i = threadIdx.x; i < MN; i += blockDim.x) {
          const float2 a = ab2[(long long)i * mcount + key];
          smat[i] = make_float4(a.x, a.x, a.y, a.y);
        }
        sa0 = wrap_cell(-svec[key] - 1, nc);
        sa1 = sa0;
        key_cur = key;
      }
    }
    __syncthreads();
    df3_pair_planar<IN_DF>(cur, D * (W / 2));
    __syncthreads();
    if (nbuf == 2 && o + ostep < o1) issue(o + ostep, raw + (b ^ 1) * bstride);

    if (active) {
      if (sa0 == sa1) df3_run<N, PERIODIC, true, OUT_DF>(cur, M, c0, cb, ce, sa0, sa1, nc, fb, rstride);
      else df3_run<N, PERIODIC, false, OUT_DF>(cur, M, c0, cb, ce, sa0, sa1, nc, fb, rstride);
    }
    __syncthreads();  // the tile (and a per-tile matrix) is rewritten next
  }
}

// Strided sweeps in the (ncols, rstride, ostride, outer) form:
//   x2: ncols = D0, rows stride D0, outer = v-planes (D2 D3), stride D0 D1;
//   v1: ncols = Dx, rows stride Dx, outer = D3, stride Dx D2;
//   v2: ncols = Dx, rows stride Dx D2, outer = D2 (the v1 index), stride Dx.
template <int N, bool IN_DF, bool OUT_DF>
cudaError_t launch_strided_df3_T(const SweepArgs& a, cudaStream_t st) {
  double* f = reinterpret_cast<double*>(a.f);
  double* out = reinterpret_cast<double*>(a.out ? a.out : a.f);
  const float2* ab2 = reinterpret_cast<const float2*>(a.ab2);
  const long long D = (long long)a.nc * N;
  const bool percol = a.dim >= 2;
  if (reinterpret_cast<uintptr_t>(out) & 15) return cudaErrorNotSupported;
  if (!percol && !a.periodic) return cudaErrorNotSupported;
  long long ncols, rstride, ostride, outer;
  if (a.dim == 3) {
    ncols = a.key_mod;
    rstride = a.inner;
    ostride = a.key_mod;
    outer = a.inner / a.key_mod;
  } else {
    ncols = a.inner;
    rstride = a.inner;
    ostride = D * a.inner;
    outer = a.outer;
  }
  if (percol && ncols != a.key_mod) return cudaErrorNotSupported;
  if ((ncols | rstride | ostride) & 1) return cudaErrorNotSupported;  // 16-byte column pairs
  if (ncols > 0x7fffffffLL - kStridedW || outer > 0x7fffffffLL || a.key_div > 0x7fffffffLL ||
      a.key_mod > 0x7fffffffLL || D * kStridedW > 0x7fffffffLL)
    return cudaErrorNotSupported;
  const long long ncolblk = (ncols + kStridedW - 1) / kStridedW;
  const int tpc = percol ? kDf3TilesPerCtaV : kDf3TilesPerCtaX;
  long long gy = (outer + tpc - 1) / tpc;
  if (gy > 65535) gy = 65535;
  const dim3 grid((unsigned)ncolblk, (unsigned)gy);
  using KFn = decltype(&k_sweep_strided_df3<N, true, true, IN_DF, OUT_DF>);
  KFn kfn;
  if (!percol) kfn = k_sweep_strided_df3<N, true, false, IN_DF, OUT_DF>;
  else kfn = a.periodic ? k_sweep_strided_df3<N, true, true, IN_DF, OUT_DF>
                        : k_sweep_strided_df3<N, false, true, IN_DF, OUT_DF>;
  // two buffers while two CTAs still fit on an SM (228 KB, 1 KB reserved each)
  int nbuf = 2;
  auto smem_of = [&](int nb) {
    return percol ? strided_df3_smem<N, true>(D, nb) : strided_df3_smem<N, false>(D, nb);
  };
  size_t smem = smem_of(nbuf);
  if (nbuf == 2 && smem > 115 * 1024) {
    nbuf = 1;
    smem = smem_of(1);
  }
  if (smem > 227 * 1024) return cudaErrorNotSupported;
  cudaError_t e = set_smem(kfn, smem);
  if (e != cudaSuccess) return e;
  kfn<<<grid, kDf3Threads, smem, st>>>(f, out, (int)ncols, rstride, ostride, a.nc, (int)outer, nbuf, ab2,
                                       a.s, a.mcount, (int)a.key_div, (int)a.key_mod);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// x1 forward sweep, FP64 storage, packed double-float.  A tile is R (even)
// consecutive lines with one matrix pair; lines 2p and 2p+1 are the two
// lanes.  A CTA walks kX1Df3TilesPerCta tiles and loads tile t+1 (cp.async)
// while it computes tile t:
//   wait for tile t; stage its matrix                     | barrier
//   convert raw t into line-pair planes ph, pl ([R/2][D]) | barrier
//   start loading tile t+1 into the other raw buffer
//   outputs of tile t into raw t (already converted)      | barrier
//   store raw t contiguously
// Thread (p, t): line pair p, cells [cb, ce) of it (a sliding window over
// the source cells, as in the strided kernel).
// ---------------------------------------------------------------------------
constexpr int kX1Df3Threads = 256;
constexpr int kX1Df3TilesPerCta = 8;
constexpr size_t kX1Df3SmemBudget = 75 * 1024;  // three CTAs per SM

template <int N>
inline size_t x1_df3_smem(long long D, int R) {
  return (size_t)(2 * N * N) * sizeof(float4) + 3 * (size_t)R * D * sizeof(double);
}

template <int N, bool IN_DF, bool OUT_DF>
__global__ void __launch_bounds__(kX1Df3Threads, 3)
    k_sweep_x1_df3(double* __restrict__ f, int nc, int R, int tpp_log2, long long ntiles,
                   const float2* __restrict__ ab2, const int* __restrict__ svec, long long mcount,
                   int key_div, int key_mod) {
  constexpr int MN = 2 * N * N;
  extern __shared__ __align__(16) unsigned char smraw[];
  float4* smat = reinterpret_cast<float4*>(smraw);
  const int D = nc * N;
  const int TL = R * D;  // doubles per tile
  double* raw0 = reinterpret_cast<double*>(smraw + MN * sizeof(float4));  // two tile buffers
  float2* ph = reinterpret_cast<float2*>(raw0 + 2 * TL);
  float2* pl = ph + TL / 2;
  const int TPP = 1 << tpp_log2;  // threads per line pair
  const int p = threadIdx.x >> tpp_log2, t = threadIdx.x & (TPP - 1);
  const int cpt = (nc + TPP - 1) >> tpp_log2;
  const int cb = min(t * cpt, nc), ce = min(cb + cpt, nc);
  const long long tile0 = (long long)blockIdx.x * kX1Df3TilesPerCta;
  const long long tile1 = min(tile0 + kX1Df3TilesPerCta, ntiles);
  const int chunks = TL / 2;

  auto issue = [&](long long tile, double* dst) {
    const double* src = f + tile * TL;
    for (int i = threadIdx.x; i < chunks; i += blockDim.x) cp_async16(dst + 2 * i, src + 2 * i);
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
  issue(tile0, raw0);
  int b = 0;
  for (long long tile = tile0; tile < tile1; ++tile, b ^= 1) {
    double* cur = raw0 + b * TL;
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    const int key = (int)(((tile * R) / key_div) % key_mod);
    for (int i = threadIdx.x; i < MN; i += blockDim.x) {
      const float2 a = ab2[(long long)i * mcount + key];
      smat[i] = make_float4(a.x, a.x, a.y, a.y);
    }
    const int sa = wrap_cell(-svec[key] - 1, nc);
    __syncthreads();
    {  // line-pair planes: ph[p][k] = (hi of line 2p, hi of line 2p+1), pl likewise
      const double* la = cur + (2 * p) * D;
      for (int k = t; k < D; k += TPP) {
        float h0, l0, h1, l1;
        load_pair<IN_DF>(la[k], h0, l0);
        load_pair<IN_DF>(la[D + k], h1, l1);
        ph[p * D + k] = make_float2(h0, h1);
        pl[p * D + k] = make_float2(l0, l1);
      }
    }
    __syncthreads();
    if (tile + 1 < tile1) issue(tile + 1, raw0 + (b ^ 1) * TL);
    if (cb < ce) {
      const float2* rh = ph + p * D;
      const float2* rl = pl + p * D;
      double* oa = cur + (2 * p) * D;
      int ka = cb + sa;
      if (ka >= nc) ka -= nc;
      float2 ah[N], al[N], bh[N], bl[N];
#pragma unroll
      for (int l = 0; l < N; ++l) {
        ah[l] = rh[ka * N + l];
        al[l] = rl[ka * N + l];
      }
#pragma unroll 1
      for (int c = cb; c < ce; ++c) {
        const int kb = ka + 1 == nc ? 0 : ka + 1;
#pragma unroll
        for (int l = 0; l < N; ++l) {
          bh[l] = rh[kb * N + l];
          bl[l] = rl[kb * N + l];
        }
        {
          float2 sh[N], sl[N];
          df3_accumulate<N>(smat, ah, al, bh, bl, sh, sl);
#pragma unroll
          for (int j = 0; j < N; ++j) {
            oa[c * N + j] = store_pair<OUT_DF>(sh[j].x, sl[j].x);
            oa[D + c * N + j] = store_pair<OUT_DF>(sh[j].y, sl[j].y);
          }
        }
#pragma unroll
        for (int l = 0; l < N; ++l) {
          ah[l] = bh[l];
          al[l] = bl[l];
        }
        ka = kb;
      }
    }
    __syncthreads();
    double2* dst = reinterpret_cast<double2*>(f + tile * TL);
    const double2* src = reinterpret_cast<const double2*>(cur);
    for (int i = threadIdx.x; i < chunks; i += blockDim.x) dst[i] = src[i];
  }
}

// x1 tiles: the largest even power-of-two R <= 32 that divides D1 (tiles
// never straddle two v1 nodes) and fits the shared-memory budget.
template <int N, bool IN_DF, bool OUT_DF>
cudaError_t launch_x1_df3_T(const SweepArgs& a, cudaStream_t st) {
  double* f = reinterpret_cast<double*>(a.f);
  const long long D = (long long)a.nc * N;
  int R = 0;
  for (int r = 2; r <= 32; r *= 2)
    if (a.key_div % r == 0 && x1_df3_smem<N>(D, r) <= kX1Df3SmemBudget) R = r;
  if (R == 0 || a.key_div > 0x7fffffffLL || a.key_mod > 0x7fffffffLL || R * D > 0x7fffffffLL)
    return cudaErrorNotSupported;
  int tpp_log2 = 0;
  while ((kX1Df3Threads >> tpp_log2) > R / 2) ++tpp_log2;  // (R/2) << tpp_log2 == threads
  const long long ntiles = a.outer / R;
  const long long blocks = (ntiles + kX1Df3TilesPerCta - 1) / kX1Df3TilesPerCta;
  if (blocks > 0x7fffffffLL) return cudaErrorNotSupported;
  const size_t smem = x1_df3_smem<N>(D, R);
  auto kfn = k_sweep_x1_df3<N, IN_DF, OUT_DF>;
  cudaError_t e = set_smem(kfn, smem);
  if (e != cudaSuccess) return e;
  kfn<<<(unsigned)blocks, kX1Df3Threads, smem, st>>>(f, a.nc, R, tpp_log2, ntiles,
                                                     reinterpret_cast<const float2*>(a.ab2), a.s,
                                                     a.mcount, (int)a.key_div, (int)a.key_mod);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// x1 forward sweep, FP64 storage, packed double-float, warp per line pair.
// Lines 2p and 2p+1 (one v1 node whenever D1 is even) are the two lanes.
// Every warp owns a run of line pairs and three private shared buffers of
// 2 D doubles: two raw buffers (the next pair is loaded by cp.async while
// the current one is computed) and one plane buffer of (hA, hB, lA, lB)
// float4 per position.  Per pair: wait for its raw data | convert to planes
// | outputs of the pair into the consumed raw buffer | copy it out.  Only
// warp-level synchronisation: warps never wait for each other.
// ---------------------------------------------------------------------------
constexpr int kX1WarpPairs = 8;  // line pairs per warp

template <int N>
__device__ __forceinline__ void x1w_load_cell(const float4* __restrict__ pl, int k,
                                              float2* xh, float2* xl) {
#pragma unroll
  for (int l = 0; l < N; ++l) {
    const float4 u = pl[k * N + l];
    xh[l] = make_float2(u.x, u.y);
    xl[l] = make_float2(u.z, u.w);
  }
}

// HALF (even N): a lane's unit of work is one half of a cell's outputs
// instead of a run of whole cells, for lines whose cell count leaves many
// lanes idle at whole cells (36 cells: 18 of 32 lanes busy, against 72
// half-cells on 32 lanes in three rounds); each unit reads both source
// cells, the whole-cell run slides over them.
template <int N, bool IN_DF, bool OUT_DF, bool HALF>
__global__ void __launch_bounds__(256, N >= 4 ? 2 : 3)
    k_sweep_x1_warp(double* __restrict__ f, int nc, long long npairs, int pairs_per_warp,
                    const float2* __restrict__ ab2, const int* __restrict__ svec, long long mcount,
                    int key_div, int key_mod) {
  constexpr int MN = 2 * N * N;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int D = nc * N;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  // per warp: matrices, then raw0 | raw1 | planes (2 D doubles each)
  const size_t wbytes = MN * sizeof(float4) + 3 * (size_t)(2 * D) * sizeof(double);
  unsigned char* wb = smraw + wib * wbytes;
  float4* smat = reinterpret_cast<float4*>(wb);
  double* raw0 = reinterpret_cast<double*>(wb + MN * sizeof(float4));
  float4* pl = reinterpret_cast<float4*>(raw0 + 4 * D);
  const long long gw = (long long)blockIdx.x * nwarps + wib;
  const long long p0 = gw * pairs_per_warp;
  const long long p1 = min(p0 + pairs_per_warp, npairs);
  const int cpl = (nc + 31) >> 5;  // cells per lane
  const int cb = min(lane * cpl, nc), ce = min(cb + cpl, nc);

  auto issue = [&](long long pair, double* dst) {
    const double* src = f + pair * 2 * D;
    for (int i = lane; i < D; i += 32) cp_async16(dst + 2 * i, src + 2 * i);  // 2 D doubles
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
  if (p0 < p1) issue(p0, raw0);
  int key_cur = -1, sa = 0;
  int bsel = 0;
  for (long long pair = p0; pair < p1; ++pair, bsel ^= 1) {
    double* cur = raw0 + bsel * 2 * D;
    if (pair + 1 < p1) {
      issue(pair + 1, raw0 + (bsel ^ 1) * 2 * D);
      asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    }
    const int key = (int)(((pair * 2) / key_div) % key_mod);
    if (key != key_cur) {  // warp-uniform
      if (lane < MN) {
        const float2 a = ab2[(long long)lane * mcount + key];
        smat[lane] = make_float4(a.x, a.x, a.y, a.y);
      }
      if (MN > 32)
        for (int i = lane + 32; i < MN; i += 32) {
          const float2 a = ab2[(long long)i * mcount + key];
          smat[i] = make_float4(a.x, a.x, a.y, a.y);
        }
      sa = wrap_cell(-svec[key] - 1, nc);
      key_cur = key;
    }
    __syncwarp();
    for (int k = lane; k < D; k += 32) {  // planes: (hA, hB, lA, lB) per position
      float h0, l0, h1, l1;
      load_pair<IN_DF>(cur[k], h0, l0);
      load_pair<IN_DF>(cur[D + k], h1, l1);
      pl[k] = make_float4(h0, h1, l0, l1);
    }
    __syncwarp();
    if constexpr (HALF) {
      constexpr int R = N / 2;
      for (int u = lane; u < 2 * nc; u += 32) {
        const int c = u >> 1, j0 = (u & 1) * R;
        int ka = c + sa;
        if (ka >= nc) ka -= nc;
        const int kb = ka + 1 == nc ? 0 : ka + 1;
        float2 ah[N], al[N], bh[N], bl[N];
        x1w_load_cell<N>(pl, ka, ah, al);
        x1w_load_cell<N>(pl, kb, bh, bl);
        float2 sh[R], sl[R];
        df3_accumulate_rows<N, R>(smat, j0, ah, al, bh, bl, sh, sl);
#pragma unroll
        for (int jj = 0; jj < R; ++jj) {
          cur[c * N + j0 + jj] = store_pair<OUT_DF>(sh[jj].x, sl[jj].x);
          cur[D + c * N + j0 + jj] = store_pair<OUT_DF>(sh[jj].y, sl[jj].y);
        }
      }
    } else if (cb < ce) {
      int ka = cb + sa;
      if (ka >= nc) ka -= nc;
      float2 ah[N], al[N], bh[N], bl[N];
      x1w_load_cell<N>(pl, ka, ah, al);
#pragma unroll 1
      for (int c = cb; c < ce; ++c) {
        const int kb = ka + 1 == nc ? 0 : ka + 1;
        x1w_load_cell<N>(pl, kb, bh, bl);
        float2 sh[N], sl[N];
        df3_accumulate<N>(smat, ah, al, bh, bl, sh, sl);
#pragma unroll
        for (int j = 0; j < N; ++j) {
          cur[c * N + j] = store_pair<OUT_DF>(sh[j].x, sl[j].x);
          cur[D + c * N + j] = store_pair<OUT_DF>(sh[j].y, sl[j].y);
        }
#pragma unroll
        for (int l = 0; l < N; ++l) {
          ah[l] = bh[l];
          al[l] = bl[l];
        }
        ka = kb;
      }
    }
    __syncwarp();
    double2* dst = reinterpret_cast<double2*>(f + pair * 2 * D);
    const double2* src = reinterpret_cast<const double2*>(cur);
    for (int i = lane; i < D; i += 32) dst[i] = src[i];
    __syncwarp();
  }
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

template <int N, bool IN_DF, bool OUT_DF>
cudaError_t launch_x1_warp_T(const SweepArgs& a, cudaStream_t st) {
  double* f = reinterpret_cast<double*>(a.f);
  const long long D = (long long)a.nc * N;
  const long long lines = a.outer;
  if ((D & 1) || (lines & 1) || (a.key_div & 1) || a.key_div > 0x7fffffffLL ||
      a.key_mod > 0x7fffffffLL)
    return cudaErrorNotSupported;
  const size_t wbytes = (size_t)(2 * N * N) * sizeof(float4) + 3 * (size_t)(2 * D) * sizeof(double);
  // three CTAs per SM share 228 KB, less 1 KB reserved per CTA
  int nwarps = 8;
  while (nwarps > 1 && nwarps * wbytes > 76800) nwarps /= 2;
  if (nwarps * wbytes > 200 * 1024) return cudaErrorNotSupported;
  const long long npairs = lines / 2;
  const long long warps = (npairs + kX1WarpPairs - 1) / kX1WarpPairs;
  const long long blocks = (warps + nwarps - 1) / nwarps;
  if (blocks > 0x7fffffffLL) return cudaErrorNotSupported;
  const size_t smem = nwarps * wbytes;
  // half-cell units when they keep clearly more lanes busy than whole cells
  const int nc = a.nc, cpl = (nc + 31) / 32, hr = (2 * nc + 31) / 32;
  const bool half = (N % 2 == 0) && 2 * cpl > 1.15 * hr;  // busy-lane fractions nc / 32 cpl vs 2 nc / 32 hr
  auto kfn = half ? k_sweep_x1_warp<N, IN_DF, OUT_DF, (N % 2 == 0)>
                  : k_sweep_x1_warp<N, IN_DF, OUT_DF, false>;
  cudaError_t e = set_smem(kfn, smem);
  if (e != cudaSuccess) return e;
  kfn<<<(unsigned)blocks, nwarps * 32, smem, st>>>(f, a.nc, npairs, kX1WarpPairs,
                                                  reinterpret_cast<const float2*>(a.ab2), a.s,
                                                  a.mcount, (int)a.key_div, (int)a.key_mod);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Shift-derivative partials of an adjoint v-sweep (double-float): for every
// column (x-node) and outer index o of the strided form,
//   sum over cells c and nodes j of  lam[c][j] (A' g[c+sa] + B' g[c+sa+1])_j,
// sa = -s-1 the forward source offset, lam the adjoint before the
// transposed sweep, g the forward input; one partial per (o, column) to
// epart[o * ncols + column], summed over o by the caller.  Both tiles are
// staged and converted to column pairs like the sweep tiles; the per-thread
// double-float partials are joined to FP64 and reduced over the cell runs in
// a fixed order.
// ---------------------------------------------------------------------------
template <int N>
inline size_t ebar_df3_smem(long long D, bool fuse = false, int nbuf = 1) {
  return (fuse ? 2 : 1) * (size_t)kDf3Pairs * df3_mat_stride<N>() * sizeof(float4) +
         2 * (size_t)nbuf * (D + N) * kStridedW * sizeof(double) +
         (size_t)kDf3Groups * kStridedW * sizeof(double);
}

// G_DF: the forward input gf holds double-float pairs instead of doubles.
// FUSE: the same CTA then applies the transposed sweep to the staged adjoint
// tile (forward form on the transposed tables tab2 / tsvec: [B^T; A^T],
// shifts -s - 1) and writes it back to lam, so the adjoint is read once for
// both.  LAM_DF: lam holds double-float pairs (read, and written by the
// fused form, in that format; instantiated with G_DF only).
template <int N, bool PERIODIC, bool G_DF, bool FUSE, bool LAM_DF>
__global__ void __launch_bounds__(kDf3Threads, N <= 2 ? 3 : 2)
    k_ebar_df3(double* lam, const double* __restrict__ gf,
               double* __restrict__ epart, int ncols, long long rstride, long long ostride, int nc,
               int outer, const float2* __restrict__ dab2, const int* __restrict__ svec,
               long long mcount, const float2* __restrict__ tab2, const int* __restrict__ tsvec,
               int nbuf) {
  constexpr int W = kStridedW;
  constexpr int MN = 2 * N * N;
  constexpr int MS = df3_mat_stride<N>();
  extern __shared__ __align__(16) unsigned char smraw[];
  float4* smat = reinterpret_cast<float4*>(smraw);
  float4* tmat = smat + (FUSE ? kDf3Pairs * MS : 0);  // transposed tables (FUSE)
  const int D = nc * N;
  const int bstride = (D + N) * W;
  // nbuf (1 or 2) pairs of tile buffers (adjoint, forward input): with two,
  // the next tile is staged by cp.async while the current one is computed
  double* bufs = reinterpret_cast<double*>(smraw + (size_t)(FUSE ? 2 : 1) * kDf3Pairs * MS *
                                                        sizeof(float4));
  double* red = bufs + 2 * nbuf * bstride;  // [groups][W]
  const int col0 = blockIdx.x * W;
  const int nvalid = min(W, ncols - col0);
  const int q = threadIdx.x % kDf3Pairs, g = threadIdx.x / kDf3Pairs;
  const int c0 = 2 * q;
  const int cb = (g * nc) / kDf3Groups, ce = ((g + 1) * nc) / kDf3Groups;
  const bool active = c0 < nvalid && cb < ce;

  for (int e = threadIdx.x; e < kDf3Pairs * MN; e += blockDim.x) {
    const int pq = e / MN, i = e - pq * MN;
    const int k0 = min(col0 + 2 * pq, ncols - 1), k1 = min(col0 + 2 * pq + 1, ncols - 1);
    const float2 a0 = dab2[(long long)i * mcount + k0], a1 = dab2[(long long)i * mcount + k1];
    smat[pq * MS + i] = make_float4(a0.x, a1.x, a0.y, a1.y);
    if (FUSE) {
      const float2 b0 = tab2[(long long)i * mcount + k0], b1 = tab2[(long long)i * mcount + k1];
      tmat[pq * MS + i] = make_float4(b0.x, b1.x, b0.y, b1.y);
    }
  }
  int sa0 = -svec[min(col0 + c0, ncols - 1)] - 1;
  int sa1 = -svec[min(col0 + c0 + 1, ncols - 1)] - 1;
  int ta0 = 0, ta1 = 0;  // a-cell offsets of the transposed sweep
  if (FUSE) {
    ta0 = -tsvec[min(col0 + c0, ncols - 1)] - 1;
    ta1 = -tsvec[min(col0 + c0 + 1, ncols - 1)] - 1;
  }
  if (PERIODIC) {
    sa0 = wrap_cell(sa0, nc);
    sa1 = wrap_cell(sa1, nc);
    ta0 = wrap_cell(ta0, nc);
    ta1 = wrap_cell(ta1, nc);
  }
  if (!PERIODIC)  // the zero-inflow cell rows of every buffer (never loaded)
    for (int i = threadIdx.x; i < 2 * nbuf * N * W; i += blockDim.x) {
      const int t = i / (N * W);
      bufs[t * bstride + D * W + (i - t * N * W)] = 0.0;
    }
  const float4* M = smat + q * MS;
  const int chunks = D * (W / 2);
  const int vchunks = nvalid / 2;
  auto row = [nc](int k) {
    if (PERIODIC) return k;
    return (unsigned)k < (unsigned)nc ? k : nc;
  };
  auto issue = [&](int o, double* xl, double* xg) {
    const long long bo = (long long)o * ostride + col0;
    for (int i = threadIdx.x; i < chunks; i += blockDim.x) {
      const int r = i / (W / 2), cq = i - r * (W / 2);
      if (cq < vchunks) {
        cp_async16(xl + r * W + 2 * cq, lam + bo + r * rstride + 2 * cq);
        cp_async16(xg + r * W + 2 * cq, gf + bo + r * rstride + 2 * cq);
      }
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
  if (nbuf == 2 && (int)blockIdx.y < outer) issue(blockIdx.y, bufs, bufs + bstride);
  int b = 0;
  for (int o = blockIdx.y; o < outer; o += gridDim.y, b ^= 1) {
    const long long base = (long long)o * ostride + col0;
    double* tl = bufs + (nbuf == 2 ? b : 0) * 2 * bstride;
    double* tg = tl + bstride;
    if (nbuf == 1) issue(o, tl, tg);
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    __syncthreads();
    df3_pair_planar<LAM_DF>(tl, D * (W / 2));
    df3_pair_planar<G_DF>(tg, D * (W / 2));
    __syncthreads();
    if (nbuf == 2 && o + (int)gridDim.y < outer)
      issue(o + gridDim.y, bufs + (b ^ 1) * 2 * bstride, bufs + (b ^ 1) * 2 * bstride + bstride);
    float2 ph = make_float2(0.0f, 0.0f), pl = make_float2(0.0f, 0.0f);  // per-lane partial
    bool first = true;
    if (active) {
      int k0 = cb + sa0, k1 = cb + sa1;
      if (PERIODIC) {
        if (k0 >= nc) k0 -= nc;
        if (k1 >= nc) k1 -= nc;
      }
      float2 ah[N], al[N], bh[N], bl[N];
      df3_load_cell<N, false>(tg, c0, row(k0), row(k1), ah, al);
#pragma unroll 1
      for (int c = cb; c < ce; ++c) {
        k0 = PERIODIC ? (k0 + 1 == nc ? 0 : k0 + 1) : k0 + 1;
        k1 = PERIODIC ? (k1 + 1 == nc ? 0 : k1 + 1) : k1 + 1;
        df3_load_cell<N, false>(tg, c0, row(k0), row(k1), bh, bl);
        float2 zh[N], zl[N];
        df3_accumulate<N>(M, ah, al, bh, bl, zh, zl);
        float2 lh[N], ll[N];
        df3_load_cell<N, true>(tl, c0, c, c, lh, ll);  // lam at cell c, both lanes
#pragma unroll
        for (int j = 0; j < N; ++j) {
          if (first) {
            df2_first(lh[j], ll[j], zh[j], zl[j], ph, pl);
            first = false;
          } else {
            df2_mac(lh[j], ll[j], zh[j], zl[j], ph, pl);
          }
        }
#pragma unroll
        for (int l = 0; l < N; ++l) {
          ah[l] = bh[l];
          al[l] = bl[l];
        }
      }
    }
    if (FUSE && active) {  // the transposed sweep from the staged adjoint, to lam
      const float4* MT = tmat + q * MS;
      if (ta0 == ta1) df3_run<N, PERIODIC, true, LAM_DF>(tl, MT, c0, cb, ce, ta0, ta1, nc, lam + base, rstride);
      else df3_run<N, PERIODIC, false, LAM_DF>(tl, MT, c0, cb, ce, ta0, ta1, nc, lam + base, rstride);
    }
    red[g * W + c0] = djoin_fast(ph.x, pl.x);
    red[g * W + c0 + 1] = djoin_fast(ph.y, pl.y);
    __syncthreads();
    if (threadIdx.x < nvalid) {
      double t = 0.0;
      for (int gg = 0; gg < kDf3Groups; ++gg) t += red[gg * W + threadIdx.x];
      epart[(long long)o * ncols + col0 + threadIdx.x] = t;
    }
    __syncthreads();
  }
}

// a.tab2, a.ts non-null: the fused form (partials, then the transposed sweep
// of the adjoint in place from the same staged tile)
template <int N>
cudaError_t launch_ebar_df3_T(const SweepArgs& a, cudaStream_t st) {
  double* lam = reinterpret_cast<double*>(a.f);
  const double* gf = reinterpret_cast<const double*>(a.g);
  const long long D = (long long)a.nc * N;
  const bool fuse = a.tab2 && a.ts;
  long long ncols, rstride, ostride, outer;
  if (a.dim == 3) {
    ncols = a.key_mod;
    rstride = a.inner;
    ostride = a.key_mod;
    outer = a.inner / a.key_mod;
  } else if (a.dim == 2) {
    ncols = a.inner;
    rstride = a.inner;
    ostride = D * a.inner;
    outer = a.outer;
  } else {
    return cudaErrorNotSupported;
  }
  // pair-format adjoints come with pair-format forward inputs; the fused
  // form writes the adjoint back in its own format
  if (a.in_df && (!a.g_df || (fuse && !a.out_df))) return cudaErrorNotSupported;
  if (!a.in_df && fuse && a.out_df) return cudaErrorNotSupported;
  if (ncols != a.key_mod || ((ncols | rstride | ostride) & 1) ||
      ((reinterpret_cast<uintptr_t>(lam) | reinterpret_cast<uintptr_t>(gf)) & 15) ||
      ncols > 0x7fffffffLL - kStridedW || outer > 0x7fffffffLL || D * kStridedW > 0x7fffffffLL)
    return cudaErrorNotSupported;
  // two buffer pairs while two CTAs still fit on an SM, else one
  int nbuf = ebar_df3_smem<N>(D, fuse, 2) <= 113 * 1024 ? 2 : 1;
  const size_t smem = ebar_df3_smem<N>(D, fuse, nbuf);
  if (smem > 113 * 1024) return cudaErrorNotSupported;
  const long long ncolblk = (ncols + kStridedW - 1) / kStridedW;
  long long gy = (outer + kDf3TilesPerCtaV - 1) / kDf3TilesPerCtaV;
  if (gy > 65535) gy = 65535;
  auto pick = [&](auto fuse_t) {
    constexpr bool F = decltype(fuse_t)::value;
    if (a.in_df)
      return a.periodic ? k_ebar_df3<N, true, true, F, true> : k_ebar_df3<N, false, true, F, true>;
    return a.periodic ? (a.g_df ? k_ebar_df3<N, true, true, F, false> : k_ebar_df3<N, true, false, F, false>)
                      : (a.g_df ? k_ebar_df3<N, false, true, F, false> : k_ebar_df3<N, false, false, F, false>);
  };
  auto kfn = fuse ? pick(std::true_type()) : pick(std::false_type());
  cudaError_t e = set_smem(kfn, smem);
  if (e != cudaSuccess) return e;
  kfn<<<dim3((unsigned)ncolblk, (unsigned)gy), kDf3Threads, smem, st>>>(
      lam, gf, a.epart, (int)ncols, rstride, ostride, a.nc, (int)outer,
      reinterpret_cast<const float2*>(a.dab2), a.s, a.mcount,
      reinterpret_cast<const float2*>(a.tab2), a.ts, nbuf);
  return cudaGetLastError();
}

}  // namespace sldg
