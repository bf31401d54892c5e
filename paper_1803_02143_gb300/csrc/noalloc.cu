// noalloc.cu -- the charge density rho(x) = sum_v w_v f[v][x] without any
// device allocation, for callers that cannot allocate (see sldg_rho_noalloc
// in include/sldg.h).  The partial sums live in a file-scope device array of
// fixed size; the weights are built per block in shared memory from the
// Gauss-Legendre rule.  Nothing here is called by the context-based path.
#include <cmath>
#include <mutex>

#include "ctx.h"
#include "dfloat.cuh"

namespace sldg {
namespace {

// 2^19 doubles (4 MiB): partial sums of up to 32 v-chunks of an x-plane.
constexpr long long kScratchDoubles = 1LL << 19;
constexpr int kMaxDevices = 64;
constexpr int kThreads = 256;

__device__ __align__(256) double g_rho_scratch[kScratchDoubles];

std::mutex g_mutex;
double* g_scratch_ptr[kMaxDevices] = {};

// Gauss-Legendre weights on [0,1] of the closed-form rules (n <= 4).
bool gl_weights(int n, double* w) {
  switch (n) {
    case 1: w[0] = 1.0; return true;
    case 2: w[0] = w[1] = 0.5; return true;
    case 3: w[0] = w[2] = 5.0 / 18.0; w[1] = 8.0 / 18.0; return true;
    case 4: {
      const double s30 = std::sqrt(30.0);
      w[0] = w[3] = (18.0 - s30) / 72.0;
      w[1] = w[2] = (18.0 + s30) / 72.0;
      return true;
    }
    default: return false;
  }
}

struct VQuad {
  int n;
  long long D2;         // v1 nodal values
  double h2, h3;        // v1, v2 cell widths
  double w[kMaxNodes];  // Gauss-Legendre weights on [0,1]
};

// Partial sums over one chunk of v-planes per blockIdx.y; the chunk's weights
// w_v1 w_v2 are formed once per block in shared memory as (hi, lo) pairs.
template <typename T>
__global__ void __launch_bounds__(kThreads)
    k_rho_partial_noalloc(const T* __restrict__ f, long long Dx, long long Dv, long long chunk,
                          VQuad q, double* __restrict__ part) {
  extern __shared__ float2 swv[];
  const long long v0 = blockIdx.y * chunk;
  long long v1 = v0 + chunk;
  if (v1 > Dv) v1 = Dv;
  for (long long v = v0 + threadIdx.x; v < v1; v += blockDim.x) {
    const long long i2 = v % q.D2, i3 = v / q.D2;
    const double w = (q.h2 * q.w[i2 % q.n]) * (q.h3 * q.w[i3 % q.n]);
    const float h = (float)w;
    swv[v - v0] = make_float2(h, (float)(w - (double)h));
  }
  __syncthreads();
  const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p >= Dx) return;
  double acc = 0.0;
  float sh = 0.0f, sl = 0.0f;
  int cnt = 0;
  for (long long v = v0; v < v1; ++v) {
    const float2 wv = swv[v - v0];
    float2 x;
    if constexpr (sizeof(T) == 8) x = dsplit(f[v * Dx + p]);
    else x = make_float2(f[v * Dx + p], 0.0f);
    df_mac(wv.x, wv.y, x, sh, sl);
    if (++cnt == 16) {  // flush the double-float partial into FP64 every 16 terms
      acc += djoin(sh, sl);
      sh = sl = 0.0f;
      cnt = 0;
    }
  }
  acc += djoin(sh, sl);
  part[blockIdx.y * Dx + p] = acc;
}

__global__ void k_rho_rows_noalloc(const double* __restrict__ part, int rows, long long cols,
                                   double* __restrict__ rho) {
  const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p >= cols) return;
  double acc = 0.0;
  for (int r = 0; r < rows; ++r) acc += part[(long long)r * cols + p];
  rho[p] = acc;
}

}  // namespace
}  // namespace sldg

extern "C" int sldg_rho_noalloc(const sldg_config* cfg, const void* f_dev, double* rho_dev,
                                void* stream) {
  using namespace sldg;
  if (!cfg || !f_dev || !rho_dev) return SLDG_ERR_BAD_PTR;
  // the configurations sldg_init accepts, and only those
  if (validate_config(cfg) != SLDG_OK) return SLDG_ERR_BAD_CONFIG;
  const int n = cfg->degree + 1;
  VQuad q;
  q.n = n;
  gl_weights(n, q.w);
  q.D2 = (long long)cfg->ncell[2] * n;
  q.h2 = (cfg->hi[2] - cfg->lo[2]) / cfg->ncell[2];
  q.h3 = (cfg->hi[3] - cfg->lo[3]) / cfg->ncell[3];
  const long long Dx = (long long)cfg->ncell[0] * n * cfg->ncell[1] * n;
  const long long Dv = q.D2 * cfg->ncell[3] * n;
  if (Dx > kScratchDoubles) return SLDG_ERR_UNSUPPORTED;  // x-plane beyond the fixed scratch

  // An error left pending by the caller's earlier work would otherwise be
  // reported as this call's launch failure: clear it first.
  cudaGetLastError();
  // One-time set-up per device: the device address of the scratch array.
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return SLDG_ERR_CUDA;
  }
  double* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_rho_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return SLDG_ERR_CUDA;
      }
      g_scratch_ptr[dev] = static_cast<double*>(p);
    }
    scratch = g_scratch_ptr[dev];
  }

  // v-chunks: at least 64 v-planes each, at most 32, within the scratch
  long long chunks = Dv / 64;
  if (chunks < 1) chunks = 1;
  if (chunks > 32) chunks = 32;
  if (chunks > kScratchDoubles / Dx) chunks = kScratchDoubles / Dx;
  const long long chunk = (Dv + chunks - 1) / chunks;
  const size_t smem = (size_t)chunk * sizeof(float2);
  if (smem > 200 * 1024) return SLDG_ERR_UNSUPPORTED;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  dim3 grid((unsigned)((Dx + kThreads - 1) / kThreads), (unsigned)chunks);
  cudaError_t e;
  if (cfg->precision == SLDG_FP64) {
    e = cudaFuncSetAttribute(k_rho_partial_noalloc<double>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
      k_rho_partial_noalloc<double><<<grid, kThreads, smem, st>>>(
          static_cast<const double*>(f_dev), Dx, Dv, chunk, q, scratch);
  } else {
    e = cudaFuncSetAttribute(k_rho_partial_noalloc<float>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
      k_rho_partial_noalloc<float><<<grid, kThreads, smem, st>>>(
          static_cast<const float*>(f_dev), Dx, Dv, chunk, q, scratch);
  }
  if (e != cudaSuccess) {  // nothing launched; leave no error pending
    cudaGetLastError();
    return SLDG_ERR_CUDA;
  }
  if (cudaGetLastError() != cudaSuccess) return SLDG_ERR_CUDA;
  k_rho_rows_noalloc<<<(unsigned)((Dx + kThreads - 1) / kThreads), kThreads, 0, st>>>(
      scratch, (int)chunks, Dx, rho_dev);
  if (cudaGetLastError() != cudaSuccess) return SLDG_ERR_CUDA;
  return SLDG_OK;
}
