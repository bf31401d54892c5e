// sweep_f32x2.cuh -- forward sweeps of FP32 storage with packed FP32x2
// arithmetic: every thread carries two lanes (two columns of a strided tile,
// or two lines of an x1 pair) in float2 registers and its matrix entries,
// one (lane 0, lane 1) pair per entry, in registers.  The organisation
// follows the double-float kernels of sweep_df3.cuh:
//   strided (x2, v1, v2): a CTA owns 64 columns and walks eight outer
//     indices with two tile buffers (the next tile loads while the current
//     one is computed); thread (q, g) owns column pair q and a run of
//     consecutive cells, sliding a window over the source cells, and writes
//     float2 rows straight to global memory;
//   x1: a warp owns a run of line pairs with private buffers and converts
//     each staged pair into (line 2p, line 2p+1) float2 planes.
#pragma once

#include "sweep_kernels.cuh"

namespace sldg {

constexpr int kF2W = 64;                      // columns per strided tile (256 B rows)
constexpr int kF2Threads = 256;
constexpr int kF2Pairs = kF2W / 2;            // 32 column pairs
constexpr int kF2Groups = kF2Threads / kF2Pairs;  // 8 cell runs
constexpr int kF2TilesPerCta = 8;

template <int N>
inline size_t strided_f2_smem(long long D) {
  return 2 * (size_t)(D + N) * kF2W * sizeof(float);  // two buffers with N zero rows
}

// y = A xa + B xb for one cell of both lanes, matrices in registers
template <int N>
__device__ __forceinline__ void f2_cell(const float2* A, const float2* B, const float2* xa,
                                        const float2* xb, float2* y) {
#pragma unroll
  for (int j = 0; j < N; ++j) {
    float2 acc = mul2(A[j * N], xa[0]);
#pragma unroll
    for (int l = 1; l < N; ++l) acc = fma2(A[j * N + l], xa[l], acc);
#pragma unroll
    for (int l = 0; l < N; ++l) acc = fma2(B[j * N + l], xb[l], acc);
    y[j] = acc;
  }
}

// Source cell of both lanes from a tile (row stride kF2W floats).  SAME:
// both lanes read cell k0 with one 8-byte load per node.
template <int N, bool SAME>
__device__ __forceinline__ void f2_load_cell(const float* __restrict__ t, int c0, int k0, int k1,
                                             float2* x) {
#pragma unroll
  for (int l = 0; l < N; ++l) {
    if (SAME) {
      x[l] = *reinterpret_cast<const float2*>(t + (k0 * N + l) * kF2W + c0);
    } else {
      x[l] = make_float2(t[(k0 * N + l) * kF2W + c0], t[(k1 * N + l) * kF2W + c0 + 1]);
    }
  }
}

template <int N, bool PERIODIC, bool SAME>
__device__ __forceinline__ void f2_run(const float* __restrict__ t, const float2* A,
                                       const float2* B, int c0, int cb, int ce, int sa0, int sa1,
                                       int nc, float* fb, long long rstride) {
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
  float2 xa[N], xb[N];
  f2_load_cell<N, SAME>(t, c0, row(k0), row(k1), xa);
  float* out = fb + c0 + (long long)cb * N * rstride;
  const long long cstep = (long long)N * rstride;
#pragma unroll 1
  for (int c = cb; c < ce; ++c, out += cstep) {
    k0 = next(k0);
    k1 = next(k1);
    f2_load_cell<N, SAME>(t, c0, row(k0), row(k1), xb);
    float2 y[N];
    f2_cell<N>(A, B, xa, xb, y);
#pragma unroll
    for (int j = 0; j < N; ++j) *reinterpret_cast<float2*>(out + j * rstride) = y[j];
#pragma unroll
    for (int l = 0; l < N; ++l) xa[l] = xb[l];
  }
}

// Strided FP32 sweep: element (o, row r, column c) at o*ostride + r*rstride
// + c; PERCOL: matrix and shift per column (key = column), else per tile
// (key = (o / key_div) % key_mod, contiguous outer indices per CTA).
template <int N, bool PERIODIC, bool PERCOL>
__global__ void __launch_bounds__(kF2Threads, 2)
    k_sweep_strided_f2(const float* f, float* out, int ncols, long long rstride, long long ostride,
                       int nc, int outer, const float* __restrict__ ab,
                       const int* __restrict__ svec, long long mcount, int key_div, int key_mod) {
  constexpr int W = kF2W;
  constexpr int NN = N * N;
  extern __shared__ __align__(16) unsigned char smraw[];
  float* raw = reinterpret_cast<float*>(smraw);
  const int D = nc * N;
  const int bstride = (D + N) * W;
  const int col0 = blockIdx.x * W;
  const int nvalid = min(W, ncols - col0);
  const int q = threadIdx.x % kF2Pairs, g = threadIdx.x / kF2Pairs;
  const int c0 = 2 * q;
  const int cb = (g * nc) / kF2Groups, ce = ((g + 1) * nc) / kF2Groups;
  const bool active = c0 < nvalid && cb < ce;

  float2 A[NN], B[NN];
  int sa0 = 0, sa1 = 0;
  auto load_mats = [&](int k0, int k1) {
#pragma unroll
    for (int i = 0; i < NN; ++i) {
      A[i] = make_float2(ab[(long long)i * mcount + k0], ab[(long long)i * mcount + k1]);
      B[i] = make_float2(ab[(long long)(NN + i) * mcount + k0], ab[(long long)(NN + i) * mcount + k1]);
    }
  };
  if (PERCOL) {
    const int k0 = min(col0 + c0, ncols - 1), k1 = min(col0 + c0 + 1, ncols - 1);
    load_mats(k0, k1);
    sa0 = -svec[k0] - 1;
    sa1 = -svec[k1] - 1;
    if (PERIODIC) {
      sa0 = wrap_cell(sa0, nc);
      sa1 = wrap_cell(sa1, nc);
    }
  }
  if (!PERIODIC)  // the zero cell, rows D .. D+N-1 of both buffers
    for (int i = threadIdx.x; i < N * W; i += blockDim.x) {
      raw[D * W + i] = 0.0f;
      raw[bstride + D * W + i] = 0.0f;
    }
  const int chunks = D * (W / 4);  // 16-byte chunks of a full tile
  const int vchunks = nvalid / 4;  // valid chunks per row
  auto issue = [&](int o, float* dst) {
    const float* src = f + (long long)o * ostride + col0;
    for (int i = threadIdx.x; i < chunks; i += blockDim.x) {
      const int r = i / (W / 4), cq = i - r * (W / 4);
      if (cq < vchunks) cp_async16(dst + r * W + 4 * cq, src + r * rstride + 4 * cq);
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
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
  if (o0 < o1) issue(o0, raw);
  int b = 0;
  for (int o = o0; o < o1; o += ostep, b ^= 1) {
    float* fb = out + (long long)o * ostride + col0;
    const float* cur = raw + b * bstride;
    if (!PERCOL) {
      const int key = (o / key_div) % key_mod;
      if (key != key_cur) {
        load_mats(key, key);
        sa0 = wrap_cell(-svec[key] - 1, nc);
        sa1 = sa0;
        key_cur = key;
      }
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    __syncthreads();
    if (o + ostep < o1) issue(o + ostep, raw + (b ^ 1) * bstride);
    if (active) {
      if (sa0 == sa1) f2_run<N, PERIODIC, true>(cur, A, B, c0, cb, ce, sa0, sa1, nc, fb, rstride);
      else f2_run<N, PERIODIC, false>(cur, A, B, c0, cb, ce, sa0, sa1, nc, fb, rstride);
    }
    __syncthreads();  // the buffer is reloaded two tiles on
  }
}

template <int N>
cudaError_t launch_strided_f2_T(const SweepArgs& a, cudaStream_t st) {
  float* f = reinterpret_cast<float*>(a.f);
  float* out = reinterpret_cast<float*>(a.out ? a.out : a.f);
  const long long D = (long long)a.nc * N;
  const bool percol = a.dim >= 2;
  if (!percol && !a.periodic) return cudaErrorNotSupported;
  if (reinterpret_cast<uintptr_t>(out) & 15) return cudaErrorNotSupported;
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
  if ((ncols | rstride | ostride) & 3) return cudaErrorNotSupported;  // 16-byte chunks
  if (reinterpret_cast<uintptr_t>(f) & 15) return cudaErrorNotSupported;
  if (ncols > 0x7fffffffLL - kF2W || outer > 0x7fffffffLL || a.key_div > 0x7fffffffLL ||
      a.key_mod > 0x7fffffffLL || (D + N) * kF2W * 2 > 0x7fffffffLL)
    return cudaErrorNotSupported;
  const size_t smem = strided_f2_smem<N>(D);
  if (smem > 113 * 1024) return cudaErrorNotSupported;  // two CTAs per SM
  const long long ncolblk = (ncols + kF2W - 1) / kF2W;
  long long gy = (outer + kF2TilesPerCta - 1) / kF2TilesPerCta;
  if (gy > 65535) gy = 65535;
  auto kfn = !percol ? k_sweep_strided_f2<N, true, false>
                     : (a.periodic ? k_sweep_strided_f2<N, true, true>
                                   : k_sweep_strided_f2<N, false, true>);
  cudaError_t e = set_smem(kfn, smem);
  if (e != cudaSuccess) return e;
  kfn<<<dim3((unsigned)ncolblk, (unsigned)gy), kF2Threads, smem, st>>>(
      f, out, (int)ncols, rstride, ostride, a.nc, (int)outer, reinterpret_cast<const float*>(a.ab), a.s,
      a.mcount, (int)a.key_div, (int)a.key_mod);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// x1 FP32 sweep, warp per line pair (lines 2p, 2p+1 share a v1 node when D1
// is even).  Per warp: two raw buffers of 2 D floats (the next pair loads by
// cp.async while the current one is computed) and one plane buffer of
// (line 2p, line 2p+1) float2 per position; outputs are staged in the
// consumed raw buffer and copied out contiguously.
// ---------------------------------------------------------------------------
constexpr int kF2X1PairsPerWarp = 8;

template <int N>
__global__ void __launch_bounds__(256, N >= 4 ? 3 : 4)
    k_sweep_x1_f2warp(float* __restrict__ f, int nc, long long npairs, int pairs_per_warp,
                      const float* __restrict__ ab, const int* __restrict__ svec,
                      long long mcount, int key_div, int key_mod) {
  constexpr int NN = N * N;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int D = nc * N;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  const size_t wbytes = 3 * (size_t)(2 * D) * sizeof(float);
  float* raw0 = reinterpret_cast<float*>(smraw + wib * wbytes);
  float2* pl = reinterpret_cast<float2*>(raw0 + 4 * D);
  const long long gw = (long long)blockIdx.x * nwarps + wib;
  const long long p0 = gw * pairs_per_warp;
  const long long p1 = min(p0 + pairs_per_warp, npairs);
  const int cpl = (nc + 31) >> 5;
  const int cb = min(lane * cpl, nc), ce = min(cb + cpl, nc);

  auto issue = [&](long long pair, float* dst) {
    const float* src = f + pair * 2 * D;
    for (int i = lane; i < D / 2; i += 32) cp_async16(dst + 4 * i, src + 4 * i);  // 2 D floats
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
  float2 A[NN], B[NN];
  int key_cur = -1, sa = 0;
  if (p0 < p1) issue(p0, raw0);
  int bsel = 0;
  for (long long pair = p0; pair < p1; ++pair, bsel ^= 1) {
    float* cur = raw0 + bsel * 2 * D;
    if (pair + 1 < p1) {
      issue(pair + 1, raw0 + (bsel ^ 1) * 2 * D);
      asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    }
    const int key = (int)(((pair * 2) / key_div) % key_mod);
    if (key != key_cur) {
#pragma unroll
      for (int i = 0; i < NN; ++i) {
        const float a = ab[(long long)i * mcount + key], bb = ab[(long long)(NN + i) * mcount + key];
        A[i] = make_float2(a, a);
        B[i] = make_float2(bb, bb);
      }
      sa = wrap_cell(-svec[key] - 1, nc);
      key_cur = key;
    }
    __syncwarp();
    for (int k = lane; k < D; k += 32) pl[k] = make_float2(cur[k], cur[D + k]);
    __syncwarp();
    if (cb < ce) {
      int ka = cb + sa;
      if (ka >= nc) ka -= nc;
      float2 xa[N], xb[N];
#pragma unroll
      for (int l = 0; l < N; ++l) xa[l] = pl[ka * N + l];
#pragma unroll 1
      for (int c = cb; c < ce; ++c) {
        const int kb = ka + 1 == nc ? 0 : ka + 1;
#pragma unroll
        for (int l = 0; l < N; ++l) xb[l] = pl[kb * N + l];
        float2 y[N];
        f2_cell<N>(A, B, xa, xb, y);
#pragma unroll
        for (int j = 0; j < N; ++j) {
          cur[c * N + j] = y[j].x;
          cur[D + c * N + j] = y[j].y;
        }
#pragma unroll
        for (int l = 0; l < N; ++l) xa[l] = xb[l];
        ka = kb;
      }
    }
    __syncwarp();
    float4* dst = reinterpret_cast<float4*>(f + pair * 2 * D);
    const float4* src = reinterpret_cast<const float4*>(cur);
    for (int i = lane; i < D / 2; i += 32) dst[i] = src[i];
    __syncwarp();
  }
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

template <int N>
cudaError_t launch_x1_f2warp_T(const SweepArgs& a, cudaStream_t st) {
  float* f = reinterpret_cast<float*>(a.f);
  const long long D = (long long)a.nc * N;
  const long long lines = a.outer;
  // 2 D floats per pair must be whole 16-byte chunks; lines pair up within a v1 node
  if ((D & 1) || (lines & 1) || (a.key_div & 1) || a.key_div > 0x7fffffffLL ||
      a.key_mod > 0x7fffffffLL || (reinterpret_cast<uintptr_t>(f) & 15))
    return cudaErrorNotSupported;
  const size_t wbytes = 3 * (size_t)(2 * D) * sizeof(float);
  int nwarps = 8;
  while (nwarps > 1 && nwarps * wbytes > 56 * 1024) nwarps /= 2;  // four CTAs per SM
  if (nwarps * wbytes > 200 * 1024) return cudaErrorNotSupported;
  const long long npairs = lines / 2;
  const long long warps = (npairs + kF2X1PairsPerWarp - 1) / kF2X1PairsPerWarp;
  const long long blocks = (warps + nwarps - 1) / nwarps;
  if (blocks > 0x7fffffffLL) return cudaErrorNotSupported;
  const size_t smem = nwarps * wbytes;
  auto kfn = k_sweep_x1_f2warp<N>;
  cudaError_t e = set_smem(kfn, smem);
  if (e != cudaSuccess) return e;
  kfn<<<(unsigned)blocks, nwarps * 32, smem, st>>>(f, a.nc, npairs, kF2X1PairsPerWarp,
                                                  reinterpret_cast<const float*>(a.ab), a.s,
                                                  a.mcount, (int)a.key_div, (int)a.key_mod);
  return cudaGetLastError();
}

template <int N>
cudaError_t launch_sweep_f2_N(const SweepArgs& a, cudaStream_t st) {
  if (a.adjoint || (a.dim == 0 && out_of_place(a))) return cudaErrorNotSupported;
  return a.dim == 0 ? launch_x1_f2warp_T<N>(a, st) : launch_strided_f2_T<N>(a, st);
}

// Packed FP32 forward sweeps for degrees 0..3 on aligned layouts;
// cudaErrorNotSupported sends the caller to the one-lane kernels.
inline cudaError_t launch_sweep_f2(const SweepArgs& a, cudaStream_t st) {
  switch (a.n) {
    case 1: return launch_sweep_f2_N<1>(a, st);
    case 2: return launch_sweep_f2_N<2>(a, st);
    case 3: return launch_sweep_f2_N<3>(a, st);
    case 4: return launch_sweep_f2_N<4>(a, st);
    default: return cudaErrorNotSupported;
  }
}

}  // namespace sldg
