// sweep_x12_df.cuh -- the fused X1, X2 half-drift pass of sweep_x12.cuh for
// FP64 storage in packed double-float arithmetic (the operations of
// sweep_df3.cuh).
#pragma once

#include <algorithm>

#include "sweep_df3.cuh"
#include "sweep_x12.cuh"

namespace sldg {

// ---------------------------------------------------------------------------
// A CTA's rows arrive as 8-byte elements (IEEE doubles, or (hi, lo) pairs
// when IN_DF); X1 (lanes = the two rows of a warp's row pair) writes its
// outputs back in place as (h_k, h_k+1, l_k, l_k+1) column pairs, which is
// the operand layout of X2 (lanes = two adjacent columns); X2 writes 8-byte
// elements to f (pairs when OUT_DF).  Matrices: (hi, hi, lo, lo) float4 per
// entry in shared memory.
//
// The cluster barrier between X1 and X2 is split: a CTA signals that its X1
// rows are final, computes the X2 outputs whose source cells all lie in its
// own rows, and only then waits for its peers before the outputs that read
// a peer's rows.  Small CTAs (128 threads, a plane over 8 of them at 192^2
// FP64 values: 37 KB each, six per SM) keep the phases of many CTAs
// interleaved on each SM.  The arithmetic of every output is unchanged.
// ---------------------------------------------------------------------------
constexpr int kX12DfThreads = 128;
constexpr int kX12DfSmemTarget = 38 * 1024;  // six CTAs per SM
__device__ __forceinline__ float4 ld_cluster_f4(unsigned addr) {
  float4 v;
  asm volatile("ld.shared::cluster.v4.f32 {%0, %1, %2, %3}, [%4];\n"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "r"(addr));
  return v;
}

// run: consecutive x2 cells of one X2 work item (one column pair)
template <int N, int CPL, bool GRP, bool IN_DF, bool OUT_DF>
__global__ void __launch_bounds__(kX12DfThreads, N >= 4 ? 4 : 6)
    k_sweep_x12_df(const double* src, double* dst, int nc0, int nc1, int cs, int run, int D2, int D3,
                   const float2* __restrict__ ab1, const int* __restrict__ s1,
                   const float2* __restrict__ ab2, const int* __restrict__ s2,
                   const double* __restrict__ fold_w, const double* __restrict__ fold_r) {
  constexpr int MN = 2 * N * N;
  extern __shared__ __align__(16) unsigned char smraw[];
  float4* m1 = reinterpret_cast<float4*>(smraw);
  float4* m2 = m1 + MN;
  double* rows = reinterpret_cast<double*>(m2 + MN);
  const int D0 = nc0 * N, D1 = nc1 * N;
  const unsigned rank = cluster_ctarank();
  const long long plane = blockIdx.x / cs;
  const int cells_per = nc1 / cs;
  const int H = cells_per * N;
  const double* fp = src + plane * (long long)D1 * D0;  // read
  double* op = dst + plane * (long long)D1 * D0;        // written (may be fp)
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;

  const int chunks = H * D0 / 2;
  {
    const double* sp = fp + (long long)rank * H * D0;
    for (int i = threadIdx.x; i < chunks; i += blockDim.x) cp_async16(rows + 2 * i, sp + 2 * i);
  }
  const int key1 = (int)(plane % D2), key2 = (int)((plane / D2) % D3);
  for (int i = threadIdx.x; i < MN; i += blockDim.x) {
    const float2 a = ab1[(long long)i * D2 + key1], b = ab2[(long long)i * D3 + key2];
    m1[i] = make_float4(a.x, a.x, a.y, a.y);
    m2[i] = make_float4(b.x, b.x, b.y, b.y);
  }
  cp_async_wait_all();
  if (fold_w) {
    // the charge-density adjoint folded in: rows += w_v rho_bar(x), each
    // thread on the chunks it copied; IEEE rows as k_rho_adj does it, pair
    // rows by a double-float sum with the split product
    const double w = fold_w[plane];
    const double* r = fold_r + (long long)rank * H * D0;
    for (int i = threadIdx.x; i < chunks; i += blockDim.x) {
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        if (IN_DF) {
          const float2 x = df_unpack(rows[2 * i + e]);
          const float2 t = dsplit(w * r[2 * i + e]);
          const float sh = x.x + t.x;
          const float bb = sh - x.x;
          float sl = (x.x - (sh - bb)) + (t.x - bb);
          sl += x.y + t.y;
          const float hh = sh + sl;
          rows[2 * i + e] = df_pack(hh, sl - (hh - sh));
        } else {
          rows[2 * i + e] = fma(w, r[2 * i + e], rows[2 * i + e]);
        }
      }
    }
  }
  __syncthreads();

  // X1 in place, a lane group per row pair (several groups per warp on short
  // lines); outputs as column pairs
  {
    const int sa = wrap_cell(-s1[key1] - 1, nc0);
    const int lpp = GRP ? x12_lanes_per_pair(nc0, CPL) : 32, G = GRP ? 32 / lpp : 1;
    const int grp = GRP ? lane / lpp : 0, gl = lane - grp * lpp;
    const unsigned gmask = GRP ? ((1u << lpp) - 1) << (grp * lpp) : 0xffffffffu;
    const int cb = min(gl * CPL, nc0), ce = min(cb + CPL, nc0);
    for (int p = wid * G + grp; p < H / 2; p += nw * G) {
      double* ra = rows + (2 * p) * D0;
      double* rb = ra + D0;
      float2 xh[CPL + 1][N], xl[CPL + 1][N];
      int k = cb + sa;
      if (k >= nc0) k -= nc0;
#pragma unroll
      for (int t = 0; t <= CPL; ++t) {
        if (cb + t <= ce) {
#pragma unroll
          for (int l = 0; l < N; ++l) {
            float h0, l0, h1, l1;
            load_pair<IN_DF>(ra[k * N + l], h0, l0);
            load_pair<IN_DF>(rb[k * N + l], h1, l1);
            xh[t][l] = make_float2(h0, h1);
            xl[t][l] = make_float2(l0, l1);
          }
        }
        k = k + 1 == nc0 ? 0 : k + 1;
      }
      __syncwarp(gmask);
      float* fa = reinterpret_cast<float*>(ra);
      float* fb = reinterpret_cast<float*>(rb);
#pragma unroll
      for (int t = 0; t < CPL; ++t) {
        const int c = cb + t;
        if (c < ce) {
          float2 sh[N], sl[N];
          df3_accumulate<N>(m1, xh[t], xl[t], xh[t + 1], xl[t + 1], sh, sl);
#pragma unroll
          for (int j = 0; j < N; ++j) {
            const int pos = c * N + j;
            const int o = (pos >> 1) * 4 + (pos & 1);  // float slot of h in its column pair
            fa[o] = sh[j].x;
            fa[o + 2] = sl[j].x;
            fb[o] = sh[j].y;
            fb[o + 2] = sl[j].y;
          }
        }
      }
      __syncwarp(gmask);
    }
  }
  __syncthreads();  // this CTA's X1 rows are final for all of its warps
  cluster_arrive();

  // X2 for the CTA's rows from column-pair operands: first the runs whose
  // source cells all lie in this CTA's rows, then (after the peers' X1) the
  // runs that read a peer's rows through distributed shared memory
  {
    const int d = -s2[key2] - 1;  // sources of output cell c: c + d, c + d + 1
    const int sa = wrap_cell(d, nc1);
    const int npairs = D0 / 2;
    const int items = npairs * ((cells_per + run - 1) / run);
    // exact quotients of small operands (< 2^16) by a 32-bit reciprocal
    const unsigned inv_np = 0xFFFFFFFFu / (unsigned)npairs + 1u;
    const unsigned inv_cp = 0xFFFFFFFFu / (unsigned)cells_per + 1u;
    auto local_load = [&](int lcell, int c0, float2* xh, float2* xl) {
#pragma unroll
      for (int l = 0; l < N; ++l) {
        const float4 u = *reinterpret_cast<const float4*>(rows + (lcell * N + l) * D0 + c0);
        xh[l] = make_float2(u.x, u.y);
        xl[l] = make_float2(u.z, u.w);
      }
    };
    auto any_load = [&](int owner, int lcell, int c0, float2* xh, float2* xl) {
      if (owner == (int)rank) {
        local_load(lcell, c0, xh, xl);
      } else {
        const unsigned base = cluster_map(rows + lcell * N * D0 + c0, (unsigned)owner);
#pragma unroll
        for (int l = 0; l < N; ++l) {
          const float4 u = ld_cluster_f4(base + (unsigned)(l * D0 * 8));
          xh[l] = make_float2(u.x, u.y);
          xl[l] = make_float2(u.z, u.w);
        }
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
        float2 ah[N], al[N], bh[N], bl[N];
        double* out = op + (long long)(cglob * N) * D0 + c0;
        if (local) {
          int k = lb + d;
          local_load(k, c0, ah, al);
#pragma unroll 1
          for (int c = lb; c < le; ++c, out += N * D0) {
            local_load(++k, c0, bh, bl);
            df3_cell<N, OUT_DF>(m2, ah, al, bh, bl, out, D0);
#pragma unroll
            for (int l = 0; l < N; ++l) {
              ah[l] = bh[l];
              al[l] = bl[l];
            }
          }
        } else {
          int k = cglob + sa;
          if (k >= nc1) k -= nc1;
          int owner = (int)__umulhi((unsigned)k, inv_cp);
          int lk = k - owner * cells_per;
          any_load(owner, lk, c0, ah, al);
#pragma unroll 1
          for (int c = lb; c < le; ++c, out += N * D0) {
            if (++lk == cells_per) {
              lk = 0;
              owner = owner + 1 == cs ? 0 : owner + 1;
            }
            any_load(owner, lk, c0, bh, bl);
            df3_cell<N, OUT_DF>(m2, ah, al, bh, bl, out, D0);
#pragma unroll
            for (int l = 0; l < N; ++l) {
              ah[l] = bh[l];
              al[l] = bl[l];
            }
          }
        }
      }
    }
  }
  cluster_sync();  // no CTA leaves while a peer may still read its rows
}

template <int N, int CPL, bool IN_DF, bool OUT_DF>
cudaError_t launch_x12_df_T(const double* f, double* out, const Grid& g, const void* ab1,
                            const int* s1, const void* ab2, const int* s2, cudaStream_t st,
                            int* shape, const double* fold_w, const double* fold_r) {
  const int nc0 = g.nc[0], nc1 = g.nc[1];
  const long long D0 = (long long)nc0 * N;
  const long long planes = g.D[2] * g.D[3];
  if (D0 % 2 || ((reinterpret_cast<uintptr_t>(f) | reinterpret_cast<uintptr_t>(out)) & 15))
    return cudaErrorNotSupported;
  const size_t mats = 2 * (size_t)(2 * N * N) * sizeof(float4);
  // the smallest cluster (2 to 8 CTAs) whose row share fits six CTAs per SM,
  // else the largest that fits one
  int cs = 0;
  for (int c = 2; c <= 8; c *= 2) {
    if (nc1 % c) continue;
    const long long H = (long long)(nc1 / c) * N;
    if (H % 2) continue;
    const long long smem = (long long)mats + H * D0 * (long long)sizeof(double);
    if (smem <= kX12DfSmemTarget) {
      cs = c;
      break;
    }
    if (smem <= 227 * 1024) cs = c;
  }
  if (cs == 0 || planes * cs > 0x7fffffffLL) return cudaErrorNotSupported;
  const int cells_per = nc1 / cs;
  const int run = std::min(2, cells_per);  // two-cell X2 work items
  const size_t smem = mats + (size_t)cells_per * N * D0 * sizeof(double);
  auto kfn = x12_lanes_per_pair(nc0, CPL) < 32 ? k_sweep_x12_df<N, CPL, true, IN_DF, OUT_DF>
                                               : k_sweep_x12_df<N, CPL, false, IN_DF, OUT_DF>;
  cudaError_t e = set_smem(kfn, smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(planes * cs));
  cfg.blockDim = dim3(kX12DfThreads);
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
                            static_cast<const float2*>(ab1), s1, static_cast<const float2*>(ab2),
                            s2, fold_w, fold_r);
}

template <int N, bool IN_DF, bool OUT_DF>
cudaError_t launch_x12_df_N(const double* f, double* out, const Grid& g, const void* ab1,
                            const int* s1, const void* ab2, const int* s2, cudaStream_t st,
                            int* shape, const double* fold_w, const double* fold_r) {
  if (g.nc[0] <= 64)
    return launch_x12_df_T<N, 2, IN_DF, OUT_DF>(f, out, g, ab1, s1, ab2, s2, st, shape, fold_w,
                                                fold_r);
  return cudaErrorNotSupported;
}

}  // namespace sldg
