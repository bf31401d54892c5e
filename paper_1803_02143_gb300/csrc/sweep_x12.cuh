// sweep_x12.cuh -- the two half drifts X1(tau/2), X2(tau/2) of FP32 storage
// fused into one pass over f: one x-plane (fixed v1, v2: D1 rows of D0
// values) per thread-block cluster of CS CTAs, each CTA holding D1/CS rows
// in shared memory.
//   1. every CTA stages its rows (cp.async, contiguous in f);
//   2. X1 in place on its rows, warp per row pair (each lane reads all the
//      source cells of its outputs into registers before the warp writes);
//   3. the CTA signals its peers that its X1 rows are final (the first half
//      of a split cluster barrier);
//   4. X2 for the CTA's own rows: first the outputs whose source rows (a few
//      rows away, periodic in x2) all lie in this CTA's shared memory, then,
//      after waiting for the peers, those that read a row across the split
//      from the owning CTA through distributed shared memory; outputs go
//      straight to f as float2 rows;
//   5. cluster barrier: no CTA leaves while a peer may still read its rows.
// f is read once and written once for both sweeps.  The arithmetic of every
// output is that of the separate packed kernels (sweep_f32x2.cuh).
#pragma once

#include <algorithm>

#include "sweep_f32x2.cuh"

namespace sldg {

constexpr int kX12Threads = 256;
constexpr int kX12Groups = 8;  // cell runs per column pair in the X2 phase

__device__ __forceinline__ unsigned cluster_ctarank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;\n" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\nbarrier.cluster.wait.acquire.aligned;\n" :::
                   "memory");
}
// the two halves of cluster_sync, for work between signalling and waiting
__device__ __forceinline__ void cluster_arrive() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() {
  asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}
// shared-memory address of the same variable in CTA `rank` of the cluster
__device__ __forceinline__ unsigned cluster_map(const void* p, unsigned rank) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  unsigned r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;\n" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
__device__ __forceinline__ float2 ld_cluster_f2(unsigned addr) {
  float2 v;
  asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];\n" : "=f"(v.x), "=f"(v.y) : "r"(addr));
  return v;
}

// Lanes given to one row pair in the X1 phase: the smallest power of two
// covering the line at cpl cells per lane (at most 32).
__host__ __device__ __forceinline__ int x12_lanes_per_pair(int nc0, int cpl) {
  const int need = (nc0 + cpl - 1) / cpl;
  int l = 1;
  while (l < need && l < 32) l *= 2;
  return l;
}

// CPL: cells of an x1 line per lane (nc0 <= 32 CPL); GRP: several lane
// groups per warp in the X1 phase (lines of at most 16 CPL cells)
// FOLD: add fold_w[v] fold_r[x] to the staged input first (the transposed
// passes of the adjoint)
template <int N, int CPL, bool GRP, bool FOLD>
__global__ void __launch_bounds__(kX12Threads, N >= 4 && CPL >= 4 ? 2 : 3)
    k_sweep_x12_f32(const float* src, float* dst, int nc0, int nc1, int cs, int run, int D2, int D3,
                    const float* __restrict__ ab1, const int* __restrict__ s1,
                    const float* __restrict__ ab2, const int* __restrict__ s2,
                    const double* __restrict__ fold_w, const double* __restrict__ fold_r) {
  constexpr int NN = N * N;
  extern __shared__ __align__(16) unsigned char smraw[];
  float* rows = reinterpret_cast<float*>(smraw);
  const int D0 = nc0 * N, D1 = nc1 * N;
  const unsigned rank = cluster_ctarank();
  const long long plane = blockIdx.x / cs;
  const int cells_per = nc1 / cs;  // x2 cells held by one CTA
  const int H = cells_per * N;     // rows held by one CTA
  const float* fp = src + plane * (long long)D1 * D0;  // read
  float* op = dst + plane * (long long)D1 * D0;        // written (may be fp)
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;

  // 1. stage rows rank*H .. rank*H + H - 1
  {
    const float* sp = fp + (long long)rank * H * D0;
    const int chunks = H * D0 / 4;
    for (int i = threadIdx.x; i < chunks; i += blockDim.x) cp_async16(rows + 4 * i, sp + 4 * i);
    cp_async_wait_all();
    if (FOLD) {
      // the charge-density adjoint folded in: rows += w_v rho_bar(x) in FP64
      // (the operation of k_rho_adj), each thread on the chunks it copied
      const double w = fold_w[plane];
      const double* r = fold_r + (long long)rank * H * D0;
      for (int i = threadIdx.x; i < chunks; i += blockDim.x)
#pragma unroll
        for (int j = 0; j < 4; ++j)
          rows[4 * i + j] = (float)fma(w, r[4 * i + j], (double)rows[4 * i + j]);
    }
  }
  const int key1 = (int)(plane % D2), key2 = (int)((plane / D2) % D3);
  __syncthreads();

  // 2. X1 in place, a group of lpp lanes per row pair (the two lanes of every
  //    FP32x2 op are the pair's two rows); short lines put several groups in
  //    one warp
  {
    float2 A[NN], B[NN];
#pragma unroll
    for (int i = 0; i < NN; ++i) {
      const float a = ab1[(long long)i * D2 + key1], b = ab1[(long long)(NN + i) * D2 + key1];
      A[i] = make_float2(a, a);
      B[i] = make_float2(b, b);
    }
    const int sa = wrap_cell(-s1[key1] - 1, nc0);
    const int lpp = GRP ? x12_lanes_per_pair(nc0, CPL) : 32, G = GRP ? 32 / lpp : 1;
    const int grp = GRP ? lane / lpp : 0, gl = lane - grp * lpp;
    const unsigned gmask = GRP ? ((1u << lpp) - 1) << (grp * lpp) : 0xffffffffu;
    const int cb = min(gl * CPL, nc0), ce = min(cb + CPL, nc0);
    for (int p = wid * G + grp; p < H / 2; p += nw * G) {
      float* ra = rows + (2 * p) * D0;
      float* rb = ra + D0;
      float2 x[CPL + 1][N];
      int k = cb + sa;
      if (k >= nc0) k -= nc0;
#pragma unroll
      for (int t = 0; t <= CPL; ++t) {
        if (cb + t <= ce) {  // source cells of outputs cb .. ce-1: cb+sa .. ce+sa
#pragma unroll
          for (int l = 0; l < N; ++l) x[t][l] = make_float2(ra[k * N + l], rb[k * N + l]);
        }
        k = k + 1 == nc0 ? 0 : k + 1;
      }
      __syncwarp(gmask);
#pragma unroll
      for (int t = 0; t < CPL; ++t) {
        const int c = cb + t;
        if (c < ce) {
          float2 y[N];
          f2_cell<N>(A, B, x[t], x[t + 1], y);
#pragma unroll
          for (int j = 0; j < N; ++j) {
            ra[c * N + j] = y[j].x;
            rb[c * N + j] = y[j].y;
          }
        }
      }
      __syncwarp(gmask);
    }
  }
  // 3. this CTA's X1 rows are final for all of its warps; its peers may read
  //    them from now on
  __syncthreads();
  cluster_arrive();

  // 4. X2 for rows rank*H .. rank*H + H - 1: first the runs of cells whose
  //    source rows all lie in this CTA, then (after the peers' X1) the runs
  //    that read a peer's rows through distributed shared memory; outputs
  //    go straight to f as float2 rows
  {
    float2 A[NN], B[NN];
#pragma unroll
    for (int i = 0; i < NN; ++i) {
      const float a = ab2[(long long)i * D3 + key2], b = ab2[(long long)(NN + i) * D3 + key2];
      A[i] = make_float2(a, a);
      B[i] = make_float2(b, b);
    }
    const int d = -s2[key2] - 1;  // sources of output cell c: c + d, c + d + 1
    const int sa = wrap_cell(d, nc1);
    const int npairs = D0 / 2;
    const int items = npairs * ((cells_per + run - 1) / run);
    // exact quotients of small operands (< 2^16) by a 32-bit reciprocal
    const unsigned inv_np = 0xFFFFFFFFu / (unsigned)npairs + 1u;
    const unsigned inv_cp = 0xFFFFFFFFu / (unsigned)cells_per + 1u;
    auto local_load = [&](int lcell, int c0, float2* xv) {
#pragma unroll
      for (int l = 0; l < N; ++l)
        xv[l] = *reinterpret_cast<const float2*>(rows + (lcell * N + l) * D0 + c0);
    };
    auto any_load = [&](int owner, int lcell, int c0, float2* xv) {
      if (owner == (int)rank) {
        local_load(lcell, c0, xv);
      } else {
        const unsigned base = cluster_map(rows + lcell * N * D0 + c0, (unsigned)owner);
#pragma unroll
        for (int l = 0; l < N; ++l) xv[l] = ld_cluster_f2(base + (unsigned)(l * D0 * 4));
      }
    };
    for (int pass = 0; pass < 2; ++pass) {
      if (pass == 1) cluster_wait();  // every peer's X1 rows are final
      for (int it = threadIdx.x; it < items; it += blockDim.x) {
        const int g = (int)__umulhi((unsigned)it, inv_np);
        const int c0 = 2 * (it - g * npairs);
        const int lb = g * run, le = min(lb + run, cells_per);
        const bool local = lb + d >= 0 && le + d <= cells_per - 1;
        if (local != (pass == 0)) continue;
        const int cglob = (int)rank * cells_per + lb;
        float2 xa[N], xb[N];
        float* out = op + (long long)(cglob * N) * D0 + c0;
        if (local) {
          int k = lb + d;
          local_load(k, c0, xa);
#pragma unroll 1
          for (int c = lb; c < le; ++c, out += N * D0) {
            local_load(++k, c0, xb);
            float2 y[N];
            f2_cell<N>(A, B, xa, xb, y);
#pragma unroll
            for (int j = 0; j < N; ++j) *reinterpret_cast<float2*>(out + j * D0) = y[j];
#pragma unroll
            for (int l = 0; l < N; ++l) xa[l] = xb[l];
          }
        } else {
          int k = cglob + sa;
          if (k >= nc1) k -= nc1;
          int owner = (int)__umulhi((unsigned)k, inv_cp);
          int lk = k - owner * cells_per;
          any_load(owner, lk, c0, xa);
#pragma unroll 1
          for (int c = lb; c < le; ++c, out += N * D0) {
            if (++lk == cells_per) {
              lk = 0;
              owner = owner + 1 == cs ? 0 : owner + 1;
            }
            any_load(owner, lk, c0, xb);
            float2 y[N];
            f2_cell<N>(A, B, xa, xb, y);
#pragma unroll
            for (int j = 0; j < N; ++j) *reinterpret_cast<float2*>(out + j * D0) = y[j];
#pragma unroll
            for (int l = 0; l < N; ++l) xa[l] = xb[l];
          }
        }
      }
    }
  }
  // 5. peers may still read these rows
  cluster_sync();
}

// Fused X1(frac) X2(frac) on FP32 storage; cudaErrorNotSupported when the
// layout does not fit (the caller then runs the two sweeps).
template <int N, int CPL>
cudaError_t launch_x12_T(const float* f, float* out, const Grid& g, const void* ab1, const int* s1,
                         const void* ab2, const int* s2, cudaStream_t st, int* shape,
                         const double* fold_w, const double* fold_r) {
  const int nc0 = g.nc[0], nc1 = g.nc[1];
  const long long D0 = (long long)nc0 * N;
  const long long planes = g.D[2] * g.D[3];
  if (D0 % 4 || ((reinterpret_cast<uintptr_t>(f) | reinterpret_cast<uintptr_t>(out)) & 15))
    return cudaErrorNotSupported;
  // the smallest cluster (a single CTA when the plane fits) whose row share
  // fits three CTAs per SM
  int cs = 0;
  for (int c = 1; c <= 8; c *= 2) {
    if (nc1 % c) continue;
    const long long H = (long long)(nc1 / c) * N;
    if (H % 2 || (H * D0) % 4) continue;
    if (H * D0 * (long long)sizeof(float) <= 75 * 1024) {
      cs = c;
      break;
    }
  }
  if (cs == 0 || planes * cs > 0x7fffffffLL) return cudaErrorNotSupported;
  const size_t smem = (size_t)(nc1 / cs) * N * D0 * sizeof(float);
  const int cells_per = nc1 / cs;
  const int run = std::max(1, (cells_per + kX12Groups - 1) / kX12Groups);  // cells per X2 item
  const bool grp = x12_lanes_per_pair(nc0, CPL) < 32;
  auto kfn = grp ? k_sweep_x12_f32<N, CPL, true, false> : k_sweep_x12_f32<N, CPL, false, false>;
  if (fold_w) kfn = grp ? k_sweep_x12_f32<N, CPL, true, true> : k_sweep_x12_f32<N, CPL, false, true>;
  cudaError_t e = set_smem(kfn, smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(planes * cs));
  cfg.blockDim = dim3(kX12Threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (shape) {
    shape[0] = cs;
    shape[1] = x12_lanes_per_pair(nc0, CPL);
  }
  return cudaLaunchKernelEx(&cfg, kfn, f, out, nc0, nc1, cs, run, (int)g.D[2], (int)g.D[3],
                            static_cast<const float*>(ab1), s1, static_cast<const float*>(ab2), s2,
                            fold_w, fold_r);
}

template <int N>
cudaError_t launch_x12_N(const float* f, float* out, const Grid& g, const void* ab1, const int* s1,
                         const void* ab2, const int* s2, cudaStream_t st, int* shape,
                         const double* fold_w, const double* fold_r) {
  const int nc0 = g.nc[0];
  if (nc0 <= 64) return launch_x12_T<N, 2>(f, out, g, ab1, s1, ab2, s2, st, shape, fold_w, fold_r);
  if (nc0 <= 128) return launch_x12_T<N, 4>(f, out, g, ab1, s1, ab2, s2, st, shape, fold_w, fold_r);
  return cudaErrorNotSupported;
}

}  // namespace sldg
