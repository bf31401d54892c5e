// fields.cu -- everything around the sweeps: the projection-matrix builder,
// the v-quadrature for rho, the spectral Poisson map and its transpose, the
// electric energy, the diagnostics, the initial values and the small adjoint
// helpers.  Reductions are two-stage with a fixed summation order, so every
// result is bit-reproducible run to run.
#include "dfloat.cuh"
#include <type_traits>

#include "fields.cuh"

namespace sldg {

// ---------------------------------------------------------------------------
// Compensated (Neumaier) accumulation.
// ---------------------------------------------------------------------------
struct KSum {
  double s, c;
};

__device__ inline void kadd(KSum& k, double x) {
  const double t = k.s + x;
  if (fabs(k.s) >= fabs(x)) k.c += (k.s - t) + x;
  else k.c += (x - t) + k.s;
  k.s = t;
}

__device__ inline void kmerge(KSum& a, const KSum& b) {
  kadd(a, b.s);
  a.c += b.c;
}

// Block-wide merge of per-thread compensated sums, fixed order: warp tree
// (xor shuffles) then warp 0 over the warp results in index order.
template <int M>
__device__ void block_ksum(KSum (&k)[M], KSum* shm /* 32*M */) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < M; ++q) {
    for (int off = 16; off > 0; off >>= 1) {
      KSum o;
      o.s = __shfl_xor_sync(0xffffffffu, k[q].s, off);
      o.c = __shfl_xor_sync(0xffffffffu, k[q].c, off);
      kmerge(k[q], o);
    }
  }
  if (lane == 0)
    for (int q = 0; q < M; ++q) shm[warp * M + q] = k[q];
  __syncthreads();
  if (threadIdx.x == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    for (int q = 0; q < M; ++q) {
      KSum t = shm[q];
      for (int w = 1; w < nw; ++w) kmerge(t, shm[w * M + q]);
      k[q] = t;
    }
  }
}

// ---------------------------------------------------------------------------
// Projection matrices (Eq. (AB-sldg)) for count shifts a_e = src[e]*dt*frac:
// x-sweeps take src = v-node coordinates, v-sweeps src = E at the x-nodes.
// ---------------------------------------------------------------------------
// NT: the node count b.n as a compile-time constant (the construction's
// loops unroll and its arrays stay in registers)
template <typename T, int NT>
__global__ void k_build_mats(long long count, const double* __restrict__ src, double dt,
                             double frac, double h, Basis b, T* __restrict__ ab,
                             T* __restrict__ dab, float2* __restrict__ ab2,
                             int* __restrict__ svec, T* __restrict__ abt,
                             float2* __restrict__ abt2, int* __restrict__ st,
                             float2* __restrict__ dab2) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= count) return;
  const double a = __dmul_rn(__dmul_rn(src[e], dt), frac);
  int s;
  double theta;
  split_shift(a, h, &s, &theta);
  double A[kMaxNodes * kMaxNodes], B[kMaxNodes * kMaxNodes];
  double dA[kMaxNodes * kMaxNodes], dB[kMaxNodes * kMaxNodes];
  build_ab<NT>(b, theta, A, B, dab ? dA : nullptr, dab ? dB : nullptr);
  constexpr int nn = NT * NT;
#pragma unroll
  for (int i = 0; i < nn; ++i) {
    ab[(long long)i * count + e] = (T)A[i];
    ab[(long long)(nn + i) * count + e] = (T)B[i];
    if (ab2) {  // (hi, lo) split: hi = A rounded to float, lo = the remainder
      const float ah = (float)A[i], bh = (float)B[i];
      ab2[(long long)i * count + e] = make_float2(ah, (float)(A[i] - (double)ah));
      ab2[(long long)(nn + i) * count + e] = make_float2(bh, (float)(B[i] - (double)bh));
    }
    if (dab) {
      dab[(long long)i * count + e] = (T)dA[i];
      dab[(long long)(nn + i) * count + e] = (T)dB[i];
      if (dab2) {
        const float ah = (float)dA[i], bh = (float)dB[i];
        dab2[(long long)i * count + e] = make_float2(ah, (float)(dA[i] - (double)ah));
        dab2[(long long)(nn + i) * count + e] = make_float2(bh, (float)(dB[i] - (double)bh));
      }
    }
    if (abt) {  // [B^T; A^T]: entry i = j n + l holds B[l][j], then A[l][j]
      const int j = i / NT, l = i - j * NT;
      const double bt = B[l * NT + j], at = A[l * NT + j];
      abt[(long long)i * count + e] = (T)bt;
      abt[(long long)(nn + i) * count + e] = (T)at;
      if (abt2) {
        const float bh = (float)bt, ah = (float)at;
        abt2[(long long)i * count + e] = make_float2(bh, (float)(bt - (double)bh));
        abt2[(long long)(nn + i) * count + e] = make_float2(ah, (float)(at - (double)ah));
      }
    }
  }
  svec[e] = s;
  if (st) st[e] = -s - 1;
}

// ---------------------------------------------------------------------------
// rho(x) = sum_v w_v f[v][x]  (Sec. 2: rho = int g dv, Gauss-Legendre in v).
// Stage 1: chunk of v-planes per blockIdx.y, one x-node per thread.
// ---------------------------------------------------------------------------
// Products w_v f are accumulated in double-float on the FP32 pipe (weights
// as (hi, lo) pairs, FP64 values split with integer operations); every 16
// terms the double-float partial is flushed into an FP64 sum, so the FP64
// pipe sees two adds per 16 values and the result keeps FP64 accuracy.
template <bool DF>
__device__ __forceinline__ float2 as_pair(float x) { return make_float2(x, 0.0f); }
template <bool DF>
__device__ __forceinline__ float2 as_pair(double x) { return DF ? df_unpack(x) : dsplit(x); }

// DF: the FP64 elements hold double-float (hi, lo) pairs
template <typename T, bool DF>
__global__ void k_rho_partial(const T* __restrict__ f, long long Dx, long long Dv, long long chunk,
                              const float2* __restrict__ wv2, double* __restrict__ part) {
  const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p >= Dx) return;
  const long long v0 = blockIdx.y * chunk;
  long long v1 = v0 + chunk;
  if (v1 > Dv) v1 = Dv;
  double acc = 0.0;
  long long v = v0;
  for (; v + 16 <= v1; v += 16) {
    T x[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) x[u] = f[(v + u) * Dx + p];
    float sh, sl;
    const float2 w0 = wv2[v];
    df_first(w0.x, w0.y, as_pair<DF>(x[0]), sh, sl);
#pragma unroll
    for (int u = 1; u < 16; ++u) {
      const float2 w = wv2[v + u];
      df_mac(w.x, w.y, as_pair<DF>(x[u]), sh, sl);
    }
    acc += djoin(sh, sl);
  }
  if (v < v1) {
    float sh = 0.0f, sl = 0.0f;
    for (; v < v1; ++v) {
      const float2 w = wv2[v];
      df_mac(w.x, w.y, as_pair<DF>(f[v * Dx + p]), sh, sl);
    }
    acc += djoin(sh, sl);
  }
  part[blockIdx.y * Dx + p] = acc;
}

__global__ void k_sum_rows(const double* __restrict__ part, int rows, long long cols,
                           double scale, double* __restrict__ out, int accumulate) {
  const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p >= cols) return;
  double acc = 0.0;
  for (int r = 0; r < rows; ++r) acc += part[(long long)r * cols + p];
  acc *= scale;
  out[p] = accumulate ? out[p] + acc : acc;
}

// ---------------------------------------------------------------------------
// Spectral Poisson map E = L rho on the Gauss-Legendre nodes (Sec. 3: the
// field solve is a Fourier transform; div E = rho - 1, curl E = 0):
//   rho_hat(m) = sum_n F1[n1][m1] F2[m2][n2] rho[n2][n1],
//   E_hat_d(m) = -i k_d m_d rho_hat(m) / |k m|^2  (m != 0),
//   E_d[n]     = Re sum_m G1[m1][n1] G2[n2][m2] E_hat_d(m),
// evaluated on the half range m1 >= 0 (rho real => E_hat Hermitian).
// ---------------------------------------------------------------------------
__device__ inline double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// The maps are small dense products.  Each kernel takes one row per block
// and sums over k for the block's outputs m with the k range split over
// KS = blockDim / cols threads per output, combined in a fixed order, so
// all SMs share the FP64 work instead of one warp per row.
struct Acc4 {
  double a, b, c, d;
};
__device__ inline Acc4 acc_add(Acc4 u, Acc4 v) { return {u.a + v.a, u.b + v.b, u.c + v.c, u.d + v.d}; }

template <class Term, class Out>
__device__ void block_split_sum(int cols, int K, Term term, Out out) {
  __shared__ Acc4 red[256];
  const int T = blockDim.x;  // <= 256
  const int KS = max(1, min(T / max(cols, 1), K));
  const int per = T / KS;
  const int mi = threadIdx.x % per, ks = threadIdx.x / per;
  for (int m0 = 0; m0 < cols; m0 += per) {
    const int m = m0 + mi;
    Acc4 acc = {0.0, 0.0, 0.0, 0.0};
    if (ks < KS && m < cols)
      for (int k = ks; k < K; k += KS) acc = acc_add(acc, term(m, k));
    if (ks < KS) red[ks * per + mi] = acc;
    __syncthreads();
    if (ks == 0 && m < cols) {
      Acc4 t = red[mi];
      for (int q = 1; q < KS; ++q) t = acc_add(t, red[q * per + mi]);
      out(m, t);
    }
    __syncthreads();
  }
}

// T[n2][m1] = sum_n1 F1[n1][m1] rho[n2][n1];  block = row n2
__global__ void k_pois_fwd_x(const double* __restrict__ rho, const double2* __restrict__ F1,
                             int D0, int M1, double2* __restrict__ T) {
  extern __shared__ double srow[];
  const int n2 = blockIdx.x;
  for (int i = threadIdx.x; i < D0; i += blockDim.x) srow[i] = rho[(long long)n2 * D0 + i];
  __syncthreads();
  block_split_sum(
      M1, D0,
      [&](int m1, int n1) {
        const double2 w = F1[(long long)n1 * M1 + m1];
        return Acc4{w.x * srow[n1], w.y * srow[n1], 0.0, 0.0};
      },
      [&](int m1, Acc4 t) { T[(long long)n2 * M1 + m1] = make_double2(t.a, t.b); });
}

// multiplier c_d(m) = -i k_d m_d / |k m|^2 as the real q with c = -i q
__device__ inline double pois_q(int d, int m1, int m2, double k0, double k1) {
  if (m1 == 0 && m2 == 0) return 0.0;
  const double a = k0 * m1, b = k1 * m2;
  return (d == 0 ? a : b) / (a * a + b * b);
}

// S_d[m2][m1] = c_d(m) rho_hat(m) with rho_hat(m) = sum_n2 F2[m2][n2] T[n2][m1];
// block = m2 (the multipliers are applied once per mode)
__global__ void k_pois_fwd_y(const double2* __restrict__ T, const double2* __restrict__ F2, int D1,
                             int K1, int M1, long long sstride, double k0, double k1,
                             double2* __restrict__ S) {
  const int mi = blockIdx.x;
  const int m2 = mi - K1;
  block_split_sum(
      M1, D1,
      [&](int m1, int n2) {
        const double2 t = cmul(F2[(long long)mi * D1 + n2], T[(long long)n2 * M1 + m1]);
        return Acc4{t.x, t.y, 0.0, 0.0};
      },
      [&](int m1, Acc4 r) {
        // c r = -i q r = (q r.y, -q r.x)
        const double q0 = pois_q(0, m1, m2, k0, k1), q1 = pois_q(1, m1, m2, k0, k1);
        S[(long long)mi * M1 + m1] = make_double2(q0 * r.b, -q0 * r.a);
        S[sstride + (long long)mi * M1 + m1] = make_double2(q1 * r.b, -q1 * r.a);
      });
}

// U_d[n2][m1] = sum_m2 G2[n2][m2] S_d[m2][m1];  block = n2
__global__ void k_pois_inv_y(const double2* __restrict__ S, const double2* __restrict__ G2,
                             int M2, int M1, long long sstride, long long ustride,
                             double2* __restrict__ U) {
  const int n2 = blockIdx.x;
  block_split_sum(
      M1, M2,
      [&](int m1, int mi) {
        const double2 g = G2[(long long)n2 * M2 + mi];
        const double2 a = cmul(g, S[(long long)mi * M1 + m1]);
        const double2 b = cmul(g, S[sstride + (long long)mi * M1 + m1]);
        return Acc4{a.x, a.y, b.x, b.y};
      },
      [&](int m1, Acc4 t) {
        U[(long long)n2 * M1 + m1] = make_double2(t.a, t.b);
        U[ustride + (long long)n2 * M1 + m1] = make_double2(t.c, t.d);
      });
}

// E_d[n2][n1] = Re U_d[n2][0] + 2 sum_{m1>=1} Re(G1[m1][n1] U_d[n2][m1]);  block = n2
__global__ void k_pois_inv_x(const double2* __restrict__ U, const double2* __restrict__ G1, int D0,
                             int M1, long long ustride, double* __restrict__ E1,
                             double* __restrict__ E2) {
  extern __shared__ double2 su[];
  const int n2 = blockIdx.x;
  for (int i = threadIdx.x; i < M1; i += blockDim.x) {
    su[i] = U[(long long)n2 * M1 + i];
    su[M1 + i] = U[ustride + (long long)n2 * M1 + i];
  }
  __syncthreads();
  block_split_sum(
      D0, M1 - 1,
      [&](int n1, int k) {
        const int m1 = k + 1;
        const double2 g = G1[(long long)m1 * D0 + n1];
        return Acc4{g.x * su[m1].x - g.y * su[m1].y, g.x * su[M1 + m1].x - g.y * su[M1 + m1].y,
                    0.0, 0.0};
      },
      [&](int n1, Acc4 t) {
        E1[(long long)n2 * D0 + n1] = su[0].x + 2.0 * t.a;
        E2[(long long)n2 * D0 + n1] = su[M1].x + 2.0 * t.b;
      });
}

// ---- transpose of the Poisson map -------------------------------------------
// V_d[n2][m1] = sum_n1 G1[m1][n1] Ebar_d[n2][n1];  block = n2
__global__ void k_pois_adj_x(const double* __restrict__ Eb1, const double* __restrict__ Eb2,
                             const double2* __restrict__ G1, int D0, int M1, long long vstride,
                             double2* __restrict__ V) {
  extern __shared__ double srow2[];
  const int n2 = blockIdx.x;
  for (int i = threadIdx.x; i < D0; i += blockDim.x) {
    srow2[i] = Eb1[(long long)n2 * D0 + i];
    srow2[D0 + i] = Eb2[(long long)n2 * D0 + i];
  }
  __syncthreads();
  block_split_sum(
      M1, D0,
      [&](int m1, int n1) {
        const double2 g = G1[(long long)m1 * D0 + n1];
        const double e1 = srow2[n1], e2 = srow2[D0 + n1];
        return Acc4{g.x * e1, g.y * e1, g.x * e2, g.y * e2};
      },
      [&](int m1, Acc4 t) {
        V[(long long)n2 * M1 + m1] = make_double2(t.a, t.b);
        V[vstride + (long long)n2 * M1 + m1] = make_double2(t.c, t.d);
      });
}

// P[m2][m1] = sum_d c_d(m) sum_n2 G2[n2][m2] V_d[n2][m1];  block = m2
__global__ void k_pois_adj_y(const double2* __restrict__ V, const double2* __restrict__ G2, int D1,
                             int K1, int M1, long long vstride, double k0, double k1,
                             double2* __restrict__ P) {
  const int mi = blockIdx.x;
  const int m2 = mi - K1;
  const int M2 = 2 * K1 + 1;
  block_split_sum(
      M1, D1,
      [&](int m1, int n2) {
        const double2 g = G2[(long long)n2 * M2 + mi];
        const double2 a = cmul(g, V[(long long)n2 * M1 + m1]);
        const double2 b = cmul(g, V[vstride + (long long)n2 * M1 + m1]);
        return Acc4{a.x, a.y, b.x, b.y};
      },
      [&](int m1, Acc4 h) {
        const double q0 = pois_q(0, m1, m2, k0, k1), q1 = pois_q(1, m1, m2, k0, k1);
        // c h = -i q h = (q h.y, -q h.x)
        P[(long long)mi * M1 + m1] = make_double2(q0 * h.b + q1 * h.d, -(q0 * h.a + q1 * h.c));
      });
}

// Y[p2][m1] = sum_m2 F2[m2][p2] P[m2][m1];  block = p2
__global__ void k_pois_adj_y2(const double2* __restrict__ P, const double2* __restrict__ F2, int D1,
                              int K1, int M1, double2* __restrict__ Y) {
  const int p2 = blockIdx.x;
  const int M2 = 2 * K1 + 1;
  block_split_sum(
      M1, M2,
      [&](int m1, int mi) {
        const double2 t = cmul(F2[(long long)mi * D1 + p2], P[(long long)mi * M1 + m1]);
        return Acc4{t.x, t.y, 0.0, 0.0};
      },
      [&](int m1, Acc4 t) { Y[(long long)p2 * M1 + m1] = make_double2(t.a, t.b); });
}

// rhobar[p2][p1] = Re sum_{m1} wt(m1) F1[p1][m1] Y[p2][m1], wt = 1 (m1 = 0), 2
__global__ void k_pois_adj_x2(const double2* __restrict__ Y, const double2* __restrict__ F1,
                              int D0, int M1, double* __restrict__ rhob) {
  extern __shared__ double2 sy[];
  const int p2 = blockIdx.x;
  for (int i = threadIdx.x; i < M1; i += blockDim.x) sy[i] = Y[(long long)p2 * M1 + i];
  __syncthreads();
  block_split_sum(
      D0, M1 - 1,
      [&](int p1, int k) {
        const int m1 = k + 1;
        const double2 w = F1[(long long)p1 * M1 + m1];
        return Acc4{w.x * sy[m1].x - w.y * sy[m1].y, 0.0, 0.0, 0.0};
      },
      [&](int p1, Acc4 t) {
        const double2 w0 = F1[(long long)p1 * M1];
        rhob[(long long)p2 * D0 + p1] = (w0.x * sy[0].x - w0.y * sy[0].y) + 2.0 * t.a;
      });
}

// ---------------------------------------------------------------------------
// Electric energy W = 1/2 sum_x w_x (E1^2 + E2^2), one block, written to out.
// ---------------------------------------------------------------------------
// counter (nullable): out is a history and W goes to out[*counter], which is
// then advanced (steps replayed from one recorded graph fill consecutive slots)
__global__ void k_energy(const double* __restrict__ E1, const double* __restrict__ E2,
                         const double* __restrict__ wx, long long Dx, double* __restrict__ out,
                         int* __restrict__ counter) {
  __shared__ KSum shm[32];
  KSum k[1] = {{0.0, 0.0}};
  for (long long p = threadIdx.x; p < Dx; p += blockDim.x)
    kadd(k[0], 0.5 * wx[p] * (E1[p] * E1[p] + E2[p] * E2[p]));
  block_ksum<1>(k, shm);
  if (threadIdx.x == 0) {
    if (counter) {
      const int i = *counter;
      out[i] = k[0].s + k[0].c;
      *counter = i + 1;
    } else {
      *out = k[0].s + k[0].c;
    }
  }
}

// ---------------------------------------------------------------------------
// Diagnostics: mass, L1, L2^2, kinetic with the 4D weight w_x * w_v.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_diag_partial(const T* __restrict__ f, Grid g, const double* __restrict__ wx,
                               const double* __restrict__ wv, const double* __restrict__ z2,
                               const double* __restrict__ z3, KSum* __restrict__ part) {
  __shared__ KSum shm[32 * 4];
  KSum k[4] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < g.N; i += stride) {
    const long long p = i % g.Dx;
    const long long v = i / g.Dx;
    const long long i2 = v % g.D[2], i3 = v / g.D[2];
    const double w = wx[p] * wv[v];
    const double x = (double)f[i];
    kadd(k[0], w * x);
    kadd(k[1], w * fabs(x));
    kadd(k[2], w * x * x);
    kadd(k[3], 0.5 * w * (z2[i2] * z2[i2] + z3[i3] * z3[i3]) * x);
  }
  block_ksum<4>(k, shm);
  if (threadIdx.x == 0)
    for (int q = 0; q < 4; ++q) part[blockIdx.x * 4 + q] = k[q];
}

__global__ void k_diag_final(const KSum* __restrict__ part, int nblocks, double* __restrict__ out) {
  if (threadIdx.x >= 4) return;
  const int q = threadIdx.x;
  KSum t = {0.0, 0.0};
  for (int b = 0; b < nblocks; ++b) kmerge(t, part[b * 4 + q]);
  out[q] = t.s + t.c;
}

// ---------------------------------------------------------------------------
// Initial values at the nodes (nodal interpolation).  1D factor tables:
//   kind 0 (Sec. 4, Eq. (iv-nl)): X = cos(k1 x1), cos(k2 x2); V = exp(-v1^2/2),
//          exp(-v2^2/2)/(2 pi); f = (1 + eps (X1 + X2)) V1 V2
//   kind 1: X = cos(k x); V1 = exp(-(v1-v0)^2/2) + exp(-(v1+v0)^2/2),
//          V2 = exp(-v2^2/2)/(4 pi); f = (1 + eps X1 + eps X2) V1 V2
//   kind 2 (Sec. 5, Eq. (iv-tsi)): X = cos(k x); V_d = exp(-(v-v0)^2/2) +
//          exp(-(v+v0)^2/2), V2 also / (8 pi); f = (1 + eps X1 X2) V1 V2
// tab layout: [X1 (D0)][X2 (D1)][V1 (D2)][V2 (D3)].
// ---------------------------------------------------------------------------
__global__ void k_init_tables(Grid g, int kind, double p1, double p2,
                              const double* __restrict__ zall, double* __restrict__ tab) {
  const long long tot = g.D[0] + g.D[1] + g.D[2] + g.D[3];
  const double pi = 3.14159265358979323846;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot;
       i += (long long)gridDim.x * blockDim.x) {
    int d = 0;
    long long j = i;
    while (j >= g.D[d]) {
      j -= g.D[d];
      ++d;
    }
    const double x = zall[i];
    double val;
    if (d == 0) val = cos(p1 * x);
    else if (d == 1) val = cos((kind == 0 ? p2 : p1) * x);
    else if (kind == 0) val = d == 2 ? exp(-x * x / 2.0) : exp(-x * x / 2.0) / (2.0 * pi);
    else if (kind == 1)
      val = d == 2 ? exp(-(x - p2) * (x - p2) / 2.0) + exp(-(x + p2) * (x + p2) / 2.0)
                   : exp(-x * x / 2.0) / (4.0 * pi);
    else {
      val = exp(-(x - p2) * (x - p2) / 2.0) + exp(-(x + p2) * (x + p2) / 2.0);
      if (d == 3) val /= 8.0 * pi;
    }
    tab[i] = val;
  }
}

// value (deriv = 0) or d/d eps (deriv = 1) of the initial value at node i
__device__ inline double init_value(const Grid& g, int kind, double eps, const double* tab,
                                    long long i, int deriv) {
  const long long i0 = i % g.D[0];
  long long r = i / g.D[0];
  const long long i1 = r % g.D[1];
  r /= g.D[1];
  const long long i2 = r % g.D[2], i3 = r / g.D[2];
  const double X1 = tab[i0], X2 = tab[g.D[0] + i1];
  const double V1 = tab[g.D[0] + g.D[1] + i2], V2 = tab[g.D[0] + g.D[1] + g.D[2] + i3];
  const double pert = kind == 2 ? X1 * X2 : X1 + X2;
  return (deriv ? pert : 1.0 + eps * pert) * V1 * V2;
}

template <typename T>
__global__ void k_init_fill(T* __restrict__ f, Grid g, int kind, double eps,
                            const double* __restrict__ tab) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < g.N;
       i += (long long)gridDim.x * blockDim.x)
    f[i] = (T)init_value(g, kind, eps, tab, i, 0);
}

template <typename T>
__global__ void k_param_grad_partial(const T* __restrict__ grad, Grid g, int kind,
                                     const double* __restrict__ tab, KSum* __restrict__ part) {
  __shared__ KSum shm[32];
  KSum k[1] = {{0.0, 0.0}};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < g.N;
       i += (long long)gridDim.x * blockDim.x)
    kadd(k[0], (double)grad[i] * init_value(g, kind, 0.0, tab, i, 1));
  block_ksum<1>(k, shm);
  if (threadIdx.x == 0) part[blockIdx.x] = k[0];
}

__global__ void k_ksum_final(const KSum* __restrict__ part, int n, double* __restrict__ out) {
  if (threadIdx.x != 0) return;
  KSum t = {0.0, 0.0};
  for (int b = 0; b < n; ++b) kmerge(t, part[b]);
  *out = t.s + t.c;
}

// ---------------------------------------------------------------------------
// Adjoint helpers.
// lam[v][x] += w_v rhobar[x]  (transpose of the v-quadrature)
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_rho_adj(T* __restrict__ lam, long long N, long long Dx,
                          const double* __restrict__ wv, const double* __restrict__ rhob) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    const long long p = i % Dx, v = i / Dx;
    lam[i] = (T)fma(wv[v], rhob[p], (double)lam[i]);  // as the fused x passes' fold
  }
}

// Ebar_d += c * w_x * E_d  (derivative of c W(E))
__global__ void k_energy_adj(double* __restrict__ Eb1, double* __restrict__ Eb2,
                             const double* __restrict__ E1, const double* __restrict__ E2,
                             const double* __restrict__ wx, long long Dx, double c) {
  const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p >= Dx) return;
  Eb1[p] += c * wx[p] * E1[p];
  Eb2[p] += c * wx[p] * E2[p];
}

__global__ void k_set_int(int* p, int v) { *p = v; }

// dst = the double-float pairs of the IEEE doubles in src (dst may be src)
__global__ void k_ieee_to_df(const double* src, double* dst, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float2 p = dsplit(src[i]);
    dst[i] = df_pack(p.x, p.y);
  }
}

// dst = the IEEE doubles of the double-float pairs in src (dst may be src)
__global__ void k_df_to_ieee(const double* src, double* dst, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float2 p = df_unpack(src[i]);
    dst[i] = djoin(p.x, p.y);
  }
}

// ===========================================================================
// Host launchers.
// ===========================================================================
static inline unsigned nblk(long long n, int t) { return (unsigned)((n + t - 1) / t); }

cudaError_t launch_build_mats(int prec, long long count, const double* src, double dt, double frac,
                              double h, const Basis& b, void* ab, void* dab, void* ab2, int* s,
                              cudaStream_t st, void* abt, void* abt2, int* sT, void* dab2) {
  if (count <= 0) return cudaSuccess;
  auto go = [&](auto nt) {
    constexpr int NT = decltype(nt)::value;
    if (prec == SLDG_FP64)
      k_build_mats<double, NT><<<nblk(count, 32), 32, 0, st>>>(count, src, dt, frac, h, b,
                                                                 (double*)ab, (double*)dab,
                                                                 (float2*)ab2, s, (double*)abt,
                                                                 (float2*)abt2, sT, (float2*)dab2);
    else
      k_build_mats<float, NT><<<nblk(count, 32), 32, 0, st>>>(count, src, dt, frac, h, b,
                                                                (float*)ab, (float*)dab, nullptr,
                                                                s, (float*)abt, nullptr, sT, nullptr);
  };
  switch (b.n) {
    case 1: go(std::integral_constant<int, 1>()); break;
    case 2: go(std::integral_constant<int, 2>()); break;
    case 3: go(std::integral_constant<int, 3>()); break;
    case 4: go(std::integral_constant<int, 4>()); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_rho(int prec, const void* f, const Grid& g, const float2* wv2, double* part,
                       int chunks, double* rho, cudaStream_t st, int* nlaunch, int df) {
  const long long chunk = (g.Dv + chunks - 1) / chunks;
  dim3 grid(nblk(g.Dx, 256), (unsigned)chunks);
  if (prec == SLDG_FP64 && df)
    k_rho_partial<double, true><<<grid, 256, 0, st>>>((const double*)f, g.Dx, g.Dv, chunk, wv2, part);
  else if (prec == SLDG_FP64)
    k_rho_partial<double, false><<<grid, 256, 0, st>>>((const double*)f, g.Dx, g.Dv, chunk, wv2, part);
  else
    k_rho_partial<float, false><<<grid, 256, 0, st>>>((const float*)f, g.Dx, g.Dv, chunk, wv2, part);
  k_sum_rows<<<nblk(g.Dx, 256), 256, 0, st>>>(part, chunks, g.Dx, 1.0, rho, 0);
  *nlaunch += 2;
  return cudaGetLastError();
}

cudaError_t launch_sum_rows(const double* part, int rows, long long cols, double scale, double* out,
                            int accumulate, cudaStream_t st) {
  k_sum_rows<<<nblk(cols, 256), 256, 0, st>>>(part, rows, cols, scale, out, accumulate);
  return cudaGetLastError();
}

cudaError_t launch_poisson(const PoissonArgs& a, const double* rho, double* E1, double* E2,
                           cudaStream_t st, int* nlaunch) {
  const int M1 = a.K0 + 1, M2 = 2 * a.K1 + 1;
  const long long us = (long long)a.D1 * M1;
  const int t1 = 256, t2 = 256;
  k_pois_fwd_x<<<a.D1, t1, a.D0 * sizeof(double), st>>>(rho, a.F1, a.D0, M1, a.T);
  const long long ss = (long long)M2 * M1;
  k_pois_fwd_y<<<M2, t1, 0, st>>>(a.T, a.F2, a.D1, a.K1, M1, ss, a.k0, a.k1, a.R);
  k_pois_inv_y<<<a.D1, t1, 0, st>>>(a.R, a.G2, M2, M1, ss, us, a.U);
  k_pois_inv_x<<<a.D1, t2, 2 * M1 * sizeof(double2), st>>>(a.U, a.G1, a.D0, M1, us, E1, E2);
  *nlaunch += 4;
  return cudaGetLastError();
}

cudaError_t launch_poisson_adj(const PoissonArgs& a, const double* Eb1, const double* Eb2,
                               double* rhob, cudaStream_t st, int* nlaunch) {
  const int M1 = a.K0 + 1, M2 = 2 * a.K1 + 1;
  const long long vs = (long long)a.D1 * M1;
  const int t1 = 256, t2 = 256;
  // V uses a.U (2 x D1 x M1), P uses a.R (M2 x M1), Y uses a.T (D1 x M1)
  k_pois_adj_x<<<a.D1, t1, 2 * a.D0 * sizeof(double), st>>>(Eb1, Eb2, a.G1, a.D0, M1, vs, a.U);
  k_pois_adj_y<<<M2, t1, 0, st>>>(a.U, a.G2, a.D1, a.K1, M1, vs, a.k0, a.k1, a.R);
  k_pois_adj_y2<<<a.D1, t1, 0, st>>>(a.R, a.F2, a.D1, a.K1, M1, a.T);
  k_pois_adj_x2<<<a.D1, t2, M1 * sizeof(double2), st>>>(a.T, a.F1, a.D0, M1, rhob);
  *nlaunch += 4;
  return cudaGetLastError();
}

cudaError_t launch_energy(const double* E1, const double* E2, const double* wx, long long Dx,
                          double* out, cudaStream_t st, int* counter) {
  k_energy<<<1, 256, 0, st>>>(E1, E2, wx, Dx, out, counter);
  return cudaGetLastError();
}

// Grid-stride kernels and two-stage reductions: four blocks per SM of the
// current device (the same count at allocation and at launch).
static int reduce_blocks() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) {
    cudaGetLastError();
    sms = 152;  // GB300
  }
  return 4 * sms;
}

size_t diag_scratch_doubles() { return (size_t)reduce_blocks() * 8 + 8; }

cudaError_t launch_diag(int prec, const void* f, const Grid& g, const double* wx, const double* wv,
                        const double* z2, const double* z3, double* scratch, double* out4,
                        cudaStream_t st, int* nlaunch) {
  const int nb = reduce_blocks();
  KSum* part = reinterpret_cast<KSum*>(scratch);
  if (prec == SLDG_FP64)
    k_diag_partial<double><<<nb, 256, 0, st>>>((const double*)f, g, wx, wv, z2, z3, part);
  else
    k_diag_partial<float><<<nb, 256, 0, st>>>((const float*)f, g, wx, wv, z2, z3, part);
  k_diag_final<<<1, 32, 0, st>>>(part, nb, out4);
  *nlaunch += 2;
  return cudaGetLastError();
}

cudaError_t launch_init(int prec, void* f, const Grid& g, int kind, const double* params,
                        const double* zall, double* tab, cudaStream_t st, int* nlaunch) {
  k_init_tables<<<8, 256, 0, st>>>(g, kind, params[1], params[2], zall, tab);
  if (prec == SLDG_FP64)
    k_init_fill<double><<<reduce_blocks() * 4, 256, 0, st>>>((double*)f, g, kind, params[0], tab);
  else
    k_init_fill<float><<<reduce_blocks() * 4, 256, 0, st>>>((float*)f, g, kind, params[0], tab);
  *nlaunch += 2;
  return cudaGetLastError();
}

cudaError_t launch_param_grad(int prec, const void* grad, const Grid& g, int kind,
                              const double* params, const double* zall, double* tab,
                              double* scratch, double* out, cudaStream_t st, int* nlaunch) {
  const int nb = reduce_blocks();
  KSum* part = reinterpret_cast<KSum*>(scratch);
  k_init_tables<<<8, 256, 0, st>>>(g, kind, params[1], params[2], zall, tab);
  if (prec == SLDG_FP64)
    k_param_grad_partial<double><<<nb, 256, 0, st>>>((const double*)grad, g, kind, tab, part);
  else
    k_param_grad_partial<float><<<nb, 256, 0, st>>>((const float*)grad, g, kind, tab, part);
  k_ksum_final<<<1, 32, 0, st>>>(part, nb, out);
  *nlaunch += 3;
  return cudaGetLastError();
}

cudaError_t launch_set_int(int* p, int v, cudaStream_t st) {
  k_set_int<<<1, 1, 0, st>>>(p, v);
  return cudaGetLastError();
}

cudaError_t launch_ieee_to_df(const void* src, void* dst, long long n, cudaStream_t st) {
  k_ieee_to_df<<<reduce_blocks() * 8, 256, 0, st>>>(static_cast<const double*>(src),
                                                    static_cast<double*>(dst), n);
  return cudaGetLastError();
}

cudaError_t launch_df_to_ieee(const void* src, void* dst, long long n, cudaStream_t st) {
  k_df_to_ieee<<<reduce_blocks() * 8, 256, 0, st>>>(static_cast<const double*>(src),
                                                    static_cast<double*>(dst), n);
  return cudaGetLastError();
}

cudaError_t launch_rho_adj(int prec, void* lam, const Grid& g, const double* wv,
                           const double* rhob, cudaStream_t st) {
  if (prec == SLDG_FP64)
    k_rho_adj<double><<<reduce_blocks() * 4, 256, 0, st>>>((double*)lam, g.N, g.Dx, wv, rhob);
  else
    k_rho_adj<float><<<reduce_blocks() * 4, 256, 0, st>>>((float*)lam, g.N, g.Dx, wv, rhob);
  return cudaGetLastError();
}

cudaError_t launch_energy_adj(double* Eb1, double* Eb2, const double* E1, const double* E2,
                              const double* wx, long long Dx, double c, cudaStream_t st) {
  k_energy_adj<<<nblk(Dx, 256), 256, 0, st>>>(Eb1, Eb2, E1, E2, wx, Dx, c);
  return cudaGetLastError();
}

}  // namespace sldg
