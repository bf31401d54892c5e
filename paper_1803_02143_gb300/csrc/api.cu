// api.cu -- the C ABI of libsldg (include/sldg.h): context life cycle,
// validation, the Gauss-Legendre basis and tables, the Strang step, the
// adjoint driver with checkpointing, and per-kernel timing.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "ctx.h"
#include "fields.cuh"

using namespace sldg;

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr size_t kMaxSmem = 227 * 1024;
constexpr size_t kX1TileBudget = 48 * 1024;    // FP32 x1 tiles
constexpr size_t kX1TileBudget64 = 56 * 1024;  // FP64 x1 tiles (two CTAs per SM)
constexpr int kTimerPairs = 8192;

// ---- Gauss-Legendre basis on [0,1] from the closed-form roots ---------------
bool make_basis(int n, Basis* b) {
  double x[kMaxNodes], w[kMaxNodes];
  switch (n) {
    case 1:
      x[0] = 0.0;
      w[0] = 2.0;
      break;
    case 2: {
      const double a = 1.0 / std::sqrt(3.0);
      x[0] = -a; x[1] = a;
      w[0] = w[1] = 1.0;
      break;
    }
    case 3: {
      const double a = std::sqrt(0.6);
      x[0] = -a; x[1] = 0.0; x[2] = a;
      w[0] = w[2] = 5.0 / 9.0;
      w[1] = 8.0 / 9.0;
      break;
    }
    case 4: {
      const double r = 2.0 / 7.0 * std::sqrt(6.0 / 5.0);
      const double a = std::sqrt(3.0 / 7.0 - r), c = std::sqrt(3.0 / 7.0 + r);
      const double s30 = std::sqrt(30.0);
      x[0] = -c; x[1] = -a; x[2] = a; x[3] = c;
      w[0] = w[3] = (18.0 - s30) / 36.0;
      w[1] = w[2] = (18.0 + s30) / 36.0;
      break;
    }
    default:
      return false;
  }
  b->n = n;
  for (int i = 0; i < n; ++i) {
    b->xi[i] = 0.5 * (1.0 + x[i]);
    b->w[i] = 0.5 * w[i];
  }
  for (int j = 0; j < n; ++j) {
    double p = 1.0;
    for (int m = 0; m < n; ++m)
      if (m != j) p *= (b->xi[j] - b->xi[m]);
    b->inv_den[j] = 1.0 / p;
  }
  for (int j = n; j < kMaxNodes; ++j) b->xi[j] = b->w[j] = b->inv_den[j] = 0.0;
  return true;
}

// ---- allocation and error helpers ------------------------------------------
template <typename P>
int dalloc(P** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  if (cudaMalloc(reinterpret_cast<void**>(p), bytes) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return SLDG_ERR_OOM;
  }
  return SLDG_OK;
}

template <typename P>
void dfree(P*& p) {
  if (p) cudaFree(reinterpret_cast<void*>(p));
  p = nullptr;
}

#define SLDG_TRY(expr)              \
  do {                              \
    int _rc = (expr);               \
    if (_rc != SLDG_OK) return _rc; \
  } while (0)

#define SLDG_CU(expr)                                 \
  do {                                                \
    cudaError_t _e = (expr);                          \
    if (_e != cudaSuccess) {                          \
      cudaGetLastError();                             \
      return SLDG_ERR_CUDA;                           \
    }                                                 \
  } while (0)

// ---- per-launch timing ---------------------------------------------------------
struct KTimer {
  sldg_ctx* c;
  int kind;
  long long n;
  size_t idx;
  bool on;
  KTimer(sldg_ctx* ctx, int k, long long nlaunch = 1) : c(ctx), kind(k), n(nlaunch), idx(0), on(false) {
    if (c->timing && c->ev_used < c->ev_kind.size()) {
      idx = c->ev_used++;
      c->ev_kind[idx] = k;
      cudaEventRecord(c->ev_pool[2 * idx], c->stream);
      on = true;
    }
  }
  ~KTimer() {
    if (on) cudaEventRecord(c->ev_pool[2 * idx + 1], c->stream);
    c->launches += n;
    if (c->timing) c->acc_n[kind] += n;
  }
};

// ---- grid helpers ------------------------------------------------------------------
double node_coord(const sldg_ctx* c, int d, long long i) {
  const int n = c->g.n;
  return c->cfg.lo[d] + ((double)(i / n) + c->basis.xi[i % n]) * c->g.h[d];
}

double node_weight(const sldg_ctx* c, int d, long long i) {
  return c->g.h[d] * c->basis.w[i % c->g.n];
}

int x1_lines_per_tile(const sldg_ctx* c) {
  const long long D0 = c->g.D[0], D1 = c->g.D[1];
  int best = 1;
  for (int R = 1; R <= 64 && R <= D1; ++R) {
    if (D1 % R) continue;
    if (sweep_smem_bytes(c->prec, 0, D0, R) <= (c->prec == SLDG_FP64 ? kX1TileBudget64 : kX1TileBudget)) best = R;
  }
  return best;
}

void free_all(sldg_ctx* c) {
  for (int d = 0; d < 4; ++d) dfree(c->d_w[d]);
  dfree(c->d_z[0]);  // coordinates are one allocation
  for (int d = 1; d < 4; ++d) c->d_z[d] = nullptr;
  dfree(c->d_wv);
  dfree(c->d_wv2);
  dfree(c->d_wx);
  auto free_set = [](MatSet* m) {
    dfree(m->ab); dfree(m->dab); dfree(m->dab2); dfree(m->ab2); dfree(m->s);
    dfree(m->abt); dfree(m->abt2); dfree(m->st);
  };
  for (int d = 0; d < 2; ++d) {
    for (int k = 0; k < sldg_ctx::kXSlots; ++k) free_set(&c->xm[d][k]);
    free_set(&c->vm[d]);
    dfree(c->d_E[d]);
    dfree(c->d_Eb[d]);
  }
  dfree(c->d_rho); dfree(c->d_part);
  dfree(c->d_F1); dfree(c->d_F2); dfree(c->d_G1); dfree(c->d_G2);
  dfree(c->d_T); dfree(c->d_R); dfree(c->d_U);
  dfree(c->d_W); dfree(c->d_diag); dfree(c->d_Wrec); dfree(c->d_rhob); dfree(c->d_epart);
  dfree(c->d_ckpool); dfree(c->d_seg); dfree(c->d_Ecap);
  for (int i = 0; i < 4; ++i) dfree(c->d_work[i]);
  dfree(c->d_alt);
  for (int i = 0; i < 4; ++i) {
    if (c->step_graph[i]) cudaGraphExecDestroy(c->step_graph[i]);
    c->step_graph[i] = nullptr;
  }
  dfree(c->d_counter);
  for (int i = 0; i < 2; ++i) {
    if (c->ev_up[i]) cudaEventDestroy(c->ev_up[i]);
    if (c->ev_free[i]) cudaEventDestroy(c->ev_free[i]);
    c->ev_up[i] = c->ev_free[i] = nullptr;
  }
  if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
  c->copy_stream = nullptr;
  if (c->h_W) cudaFreeHost(c->h_W);
  c->h_W = nullptr;
  c->h_W_cap = 0;
  for (auto& e : c->ev_pool) cudaEventDestroy(e);
  c->ev_pool.clear();
}

PoissonArgs poisson_args(sldg_ctx* c) {
  PoissonArgs a;
  a.D0 = (int)c->g.D[0];
  a.D1 = (int)c->g.D[1];
  a.K0 = c->K[0];
  a.K1 = c->K[1];
  a.k0 = c->kap[0];
  a.k1 = c->kap[1];
  a.F1 = c->d_F1; a.F2 = c->d_F2; a.G1 = c->d_G1; a.G2 = c->d_G2;
  a.T = c->d_T; a.R = c->d_R; a.U = c->d_U;
  return a;
}

// ---- matrices -------------------------------------------------------------------
int alloc_matset(sldg_ctx* c, MatSet* m, long long count, bool deriv, bool trans) {
  const size_t nn = (size_t)c->g.n * c->g.n;
  if (!m->ab) {
    SLDG_TRY(dalloc(&m->ab, 2 * nn * count * c->esize));
    SLDG_TRY(dalloc(&m->s, count * sizeof(int)));
    if (c->prec == SLDG_FP64) SLDG_TRY(dalloc(&m->ab2, 2 * nn * count * sizeof(float2)));
    m->count = count;
  }
  if (deriv && !m->dab) {
    SLDG_TRY(dalloc(&m->dab, 2 * nn * count * c->esize));
    if (c->prec == SLDG_FP64) SLDG_TRY(dalloc(&m->dab2, 2 * nn * count * sizeof(float2)));
  }
  if (trans && !m->abt) {
    SLDG_TRY(dalloc(&m->abt, 2 * nn * count * c->esize));
    SLDG_TRY(dalloc(&m->st, count * sizeof(int)));
    if (c->prec == SLDG_FP64) SLDG_TRY(dalloc(&m->abt2, 2 * nn * count * sizeof(float2)));
  }
  return SLDG_OK;
}

bool spline(const sldg_ctx* c) { return (c->cfg.flags & SLDG_FLAG_SPLINE) != 0; }

// FP64 storage swept in double-float arithmetic, whose states between the
// stages of a step are (hi, lo) pairs
bool df_states(const sldg_ctx* c) {
  return c->prec == SLDG_FP64 && !(c->cfg.flags & (SLDG_FLAG_NATIVE_FP64 | SLDG_FLAG_SPLINE));
}

void drop_step_graphs(sldg_ctx* c) {
  for (int i = 0; i < 4; ++i) {
    if (c->step_graph[i]) cudaGraphExecDestroy(c->step_graph[i]);
    c->step_graph[i] = nullptr;
  }
}

// x-sweep d (0 or 1): one matrix pair per node of v_{d+1}, shift v dt frac,
// in one of a few slots per direction (one per shift fraction in use); trans:
// also the transposed tables of the adjoint.  Reusing a slot for another
// fraction drops the recorded step graphs, which read the slots' matrices.
int ensure_xmats(sldg_ctx* c, int d, double frac, bool trans, MatSet** out) {
  MatSet* slots = c->xm[d];
  int k = -1;
  for (int i = 0; i < sldg_ctx::kXSlots && k < 0; ++i)
    if (slots[i].valid && slots[i].frac == frac) k = i;
  if (k >= 0 && (!trans || slots[k].with_t)) {
    *out = &slots[k];
    return SLDG_OK;
  }
  if (k < 0) {
    for (int i = 0; i < sldg_ctx::kXSlots && k < 0; ++i)
      if (!slots[i].valid) k = i;
    if (k < 0) {
      k = c->xm_next[d];
      c->xm_next[d] = (k + 1) % sldg_ctx::kXSlots;
      drop_step_graphs(c);
    }
  }
  MatSet& m = slots[k];
  m.valid = false;
  *out = &m;
  const int vd = d + 2;
  SLDG_TRY(alloc_matset(c, &m, c->g.D[vd], false, trans));
  KTimer t(c, SLDG_K_VMAT);
  if (spline(c))
    SLDG_CU(launch_spline_shifts(c->prec, m.count, c->d_z[vd], c->g.dt, frac, c->g.h[d], m.ab,
                                 m.s, c->stream));
  else
    SLDG_CU(launch_build_mats(c->prec, m.count, c->d_z[vd], c->g.dt, frac, c->g.h[d], c->basis,
                              m.ab, nullptr, m.ab2, m.s, c->stream, trans ? m.abt : nullptr,
                              trans ? m.abt2 : nullptr, trans ? m.st : nullptr));
  m.frac = frac;
  m.valid = true;
  m.with_t = trans;
  return SLDG_OK;
}

// v-sweep d (0 or 1 for v1, v2): one pair per x-node, shift E_d dt frac
int ensure_vmats(sldg_ctx* c, int d, double frac, bool deriv, bool trans = false) {
  MatSet& m = c->vm[d];
  if (!c->have_field) return SLDG_ERR_STATE;
  if (m.valid && m.frac == frac && (!deriv || m.with_deriv) && (!trans || m.with_t)) return SLDG_OK;
  SLDG_TRY(alloc_matset(c, &m, c->g.Dx, deriv, trans));
  KTimer t(c, SLDG_K_VMAT);
  if (spline(c)) {
    SLDG_CU(launch_spline_shifts(c->prec, m.count, c->d_E[d], c->g.dt, frac, c->g.h[d + 2], m.ab,
                                 m.s, c->stream));
    m.frac = frac;
    m.valid = true;
    m.with_deriv = false;
    m.with_t = false;
    return SLDG_OK;
  }
  SLDG_CU(launch_build_mats(c->prec, m.count, c->d_E[d], c->g.dt, frac, c->g.h[d + 2], c->basis,
                            m.ab, deriv ? m.dab : nullptr, m.ab2, m.s, c->stream,
                            trans ? m.abt : nullptr, trans ? m.abt2 : nullptr,
                            trans ? m.st : nullptr, deriv ? m.dab2 : nullptr));
  m.frac = frac;
  m.valid = true;
  m.with_deriv = deriv;
  m.with_t = trans;
  return SLDG_OK;
}

void invalidate_vmats(sldg_ctx* c) { c->vm[0].valid = c->vm[1].valid = false; }

// ---- sweeps ---------------------------------------------------------------------------
// in_df / out_df: FP64 double-float sweeps read / write (hi, lo) pairs
// out (nullable): outputs to out and buf left unchanged (kernels that write
// in place only run on out after a copy).  g_df: gfwd holds double-float
// pairs (FP64 contexts) instead of IEEE doubles.
int run_sweep(sldg_ctx* c, void* buf, int dim, double frac, bool adjoint, const void* gfwd,
              double* Ebar, bool in_df = false, bool out_df = false, void* out = nullptr,
              bool g_df = false) {
  const Grid& g = c->g;
  if (spline(c) && adjoint) return SLDG_ERR_UNSUPPORTED;
  SweepArgs a;
  std::memset(&a, 0, sizeof(a));
  a.f = buf;
  a.out = out;
  a.g_df = g_df ? 1 : 0;
  a.prec = c->prec;
  a.n = g.n;
  a.dim = dim;
  a.nc = g.nc[dim];
  a.adjoint = adjoint ? 1 : 0;
  const bool ebar = adjoint && dim >= 2 && gfwd && Ebar;
  const bool native = (c->cfg.flags & SLDG_FLAG_NATIVE_FP64) != 0;
  // a transposed sweep without the shift derivative runs the forward kernels
  // on the transposed tables ([B^T; A^T], shift entries -s - 1)
  // FP64 double-float: the shift derivative is a separate kernel on the
  // adjoint before the sweep, and the sweep itself runs in forward form
  const bool ebar_df = ebar && c->prec == SLDG_FP64 && !native;
  const bool tform = adjoint && (!ebar || ebar_df) && !(c->prec == SLDG_FP64 && native);
  MatSet* m;
  if (dim < 2) {
    SLDG_TRY(ensure_xmats(c, dim, frac, tform, &m));
    a.periodic = 1;
  } else {
    SLDG_TRY(ensure_vmats(c, dim - 2, frac, ebar, tform));
    m = &c->vm[dim - 2];
    a.periodic = g.vbc == SLDG_VBC_PERIODIC;
  }
  a.ab = tform ? m->abt : m->ab;
  a.ab2 = tform ? m->abt2 : m->ab2;
  a.dab = m->dab;
  a.dab2 = m->dab2;
  a.native_fp64 = native ? 1 : 0;
  a.in_df = in_df ? 1 : 0;
  a.out_df = out_df ? 1 : 0;
  a.s = tform ? m->st : m->s;
  a.mcount = m->count;
  if (tform) a.adjoint = 0;
  switch (dim) {
    case 0:
      a.inner = 1;
      a.outer = g.N / g.D[0];
      a.key_div = g.D[1];
      a.key_mod = g.D[2];
      a.lines_per_tile = x1_lines_per_tile(c);
      break;
    case 1:
      a.inner = g.D[0];
      a.outer = g.D[2] * g.D[3];
      a.key_div = g.D[2];
      a.key_mod = g.D[3];
      break;
    case 2:
      a.inner = g.Dx;
      a.outer = g.D[3];
      a.key_div = 1;
      a.key_mod = g.Dx;
      break;
    default:
      a.inner = g.Dx * g.D[2];
      a.outer = 1;
      a.key_div = 1;
      a.key_mod = g.Dx;
      break;
  }
  if (ebar) {
    a.g = gfwd;
    a.epart = c->d_epart;
  }
  const int kind = adjoint ? (dim < 2 ? SLDG_K_ADJ_X : SLDG_K_ADJ_V) : SLDG_K_X1 + dim;
  bool swept = false;      // the transposed sweep ran with the partials
  bool lam_to_df = false;  // the IEEE fallback's result goes back to pairs
  if (ebar_df) {  // partials of d/dE <lam, S g> from the adjoint before the sweep
    KTimer t(c, kind);
    SweepArgs ae = a;
    ae.s = m->s;  // the forward shifts (a carries the transposed form)
    ae.tab2 = m->abt2;  // and the transposed sweep from the same staged tile
    ae.ts = m->st;
    cudaError_t e = out_of_place(a) ? cudaErrorNotSupported : launch_ebar_df(ae, c->stream);
    swept = e == cudaSuccess;
    if (e == cudaErrorNotSupported) {  // the partials alone, the sweep separately
      ae.tab2 = nullptr;
      ae.ts = nullptr;
      e = launch_ebar_df(ae, c->stream);
    }
    if (e == cudaErrorNotSupported) {  // layout not taken: the fused FP64 FMA kernel
      t.n = 0;
      a.ab = m->ab;
      a.ab2 = m->ab2;
      a.s = m->s;
      a.adjoint = 1;
      if (a.g_df) {  // that kernel reads the forward input as IEEE doubles
        SLDG_CU(launch_df_to_ieee(gfwd, const_cast<void*>(gfwd), g.N, c->stream));
        c->launches += 1;
        a.g_df = 0;
      }
      if (a.in_df) {  // and the adjoint too, which it writes back as doubles
        SLDG_CU(launch_df_to_ieee(buf, buf, g.N, c->stream));
        c->launches += 1;
      }
      lam_to_df = a.out_df != 0;
      a.in_df = 0;
      a.out_df = 0;
    } else if (e != cudaSuccess) {
      cudaGetLastError();
      return SLDG_ERR_CUDA;
    }
  }
  if (!swept) {
    auto launch = [&](const SweepArgs& x) {
      if (spline(c)) return launch_spline_sweep(x, c->stream);
      if (c->prec == SLDG_FP32) return launch_sweep_f32(x, c->stream);
      if (x.adjoint || x.native_fp64) return launch_sweep_f64(x, c->stream);
      return launch_sweep_df(x, c->stream);
    };
    KTimer t(c, kind);
    cudaError_t e = launch(a);
    if (e == cudaErrorNotSupported && out_of_place(a)) {  // in place on a copy
      SLDG_CU(cudaMemcpyAsync(a.out, a.f, g.N * c->esize, cudaMemcpyDeviceToDevice, c->stream));
      a.f = a.out;
      a.out = nullptr;
      e = launch(a);
    }
    if (e != cudaSuccess) {
      cudaGetLastError();
      return SLDG_ERR_CUDA;
    }
  }
  if (lam_to_df) {
    SLDG_CU(launch_ieee_to_df(buf, buf, g.N, c->stream));
    c->launches += 1;
  }
  if (ebar) {
    // Ebar[x] += dt*frac/h_v * sum over the rows of partials at x
    const long long rows = dim == 2 ? g.D[3] : g.D[2];
    KTimer t(c, SLDG_K_OTHER);
    SLDG_CU(launch_sum_rows(c->d_epart, (int)rows, g.Dx, g.dt * frac / g.h[dim], Ebar, 1,
                            c->stream));
  }
  return SLDG_OK;
}

int compute_fields(sldg_ctx* c, const void* buf, bool df = false) {
  int nl = 0;
  {
    KTimer t(c, SLDG_K_RHO, 2);
    SLDG_CU(launch_rho(c->prec, buf, c->g, c->d_wv2, c->d_part, c->rho_chunks, c->d_rho, c->stream,
                       &nl, df ? 1 : 0));
  }
  {
    KTimer t(c, SLDG_K_POISSON, 4);
    nl = 0;
    SLDG_CU(launch_poisson(poisson_args(c), c->d_rho, c->d_E[0], c->d_E[1], c->stream, &nl));
  }
  c->have_field = true;
  invalidate_vmats(c);
  return SLDG_OK;
}

// X1(frac tau) X2(frac tau) as one fused pass over each x-plane (FP32 storage,
// or FP64 storage in double-float arithmetic); *done stays false when the
// layout does not suit it and the two sweeps must run separately.
// trans: the transposed sweeps X1^T then X2^T (the adjoint of the pair, which
// commute like X1 and X2), run in forward form on the transposed tables
// ([B^T; A^T], shift entries -s - 1) like the separate adjoint x-sweeps
// out (nullable): the result goes there and buf is left unchanged
int run_x12(sldg_ctx* c, void* buf, double frac, bool in_df, bool out_df, bool* done,
            bool trans = false, void* out = nullptr, bool rho_fold = false) {
  *done = false;
  if (c->cfg.flags & (SLDG_FLAG_NO_XFUSION | SLDG_FLAG_NATIVE_FP64 | SLDG_FLAG_SPLINE))
    return SLDG_OK;
  MatSet *m0, *m1;
  SLDG_TRY(ensure_xmats(c, 0, frac, trans, &m0));
  SLDG_TRY(ensure_xmats(c, 1, frac, trans, &m1));
  const int* s0 = trans ? m0->st : m0->s;
  const int* s1 = trans ? m1->st : m1->s;
  KTimer t(c, trans ? SLDG_K_ADJ_X : SLDG_K_X12);
  const double* fw = rho_fold ? c->d_wv : nullptr;
  const double* fr = rho_fold ? c->d_rhob : nullptr;
  const cudaError_t e =
      c->prec == SLDG_FP32
          ? launch_sweep_x12_f32(buf, c->g, trans ? m0->abt : m0->ab, s0,
                                 trans ? m1->abt : m1->ab, s1, c->stream, c->x12_shape, out, fw,
                                 fr)
          : launch_sweep_x12_df(buf, c->g, trans ? m0->abt2 : m0->ab2, s0,
                                trans ? m1->abt2 : m1->ab2, s1, in_df ? 1 : 0, out_df ? 1 : 0,
                                c->stream, c->x12_shape, out, fw, fr);
  if (e == cudaErrorNotSupported) {
    t.n = 0;  // nothing launched
    return SLDG_OK;
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return SLDG_ERR_CUDA;
  }
  *done = true;
  return SLDG_OK;
}

// X1(frac tau) X2(frac tau): the fused pass, or the two sweeps; out
// (nullable): the result goes there and buf is left unchanged
int drift(sldg_ctx* c, void* buf, double frac, bool in_df, bool out_df, void* out = nullptr) {
  const bool df = in_df || out_df;
  bool fused = false;
  SLDG_TRY(run_x12(c, buf, frac, in_df, out_df, &fused, false, out));
  if (!fused) {
    void* w = buf;
    if (out && out != buf) {
      SLDG_CU(cudaMemcpyAsync(out, buf, c->g.N * c->esize, cudaMemcpyDeviceToDevice, c->stream));
      w = out;
    }
    SLDG_TRY(run_sweep(c, w, 0, frac, false, nullptr, nullptr, in_df, df));
    SLDG_TRY(run_sweep(c, w, 1, frac, false, nullptr, nullptr, df, out_df));
  }
  return SLDG_OK;
}

// ---- splitting compositions -------------------------------------------------------
// A step is a list of stages: drifts (X1 X2 by frac tau) and kicks (the
// field of the current rho, then V1 V2 by frac tau).  Order 2 is the Strang
// step of Sec. 2, D(1/2) K(1) D(1/2).  Order 4 (SLDG_FLAG_ORDER4) is the
// triple jump S(w1 tau) S(w0 tau) S(w1 tau) of Strang steps with Yoshida's
// weights w1 = 1/(2 - 2^(1/3)), w0 = 1 - 2 w1.  Merged drifts
// (SLDG_FLAG_MERGE_DRIFTS) join the drift that ends one Strang sub-step and
// the drift that starts the next.
struct Stage {
  bool kick;
  bool W;  // the first kick of a step: W of its field is recorded
  double frac;
};

int strang_weights(const sldg_ctx* c, double* w) {
  if (c->cfg.flags & SLDG_FLAG_ORDER4) {
    w[0] = w[2] = 1.0 / (2.0 - std::cbrt(2.0));
    w[1] = 1.0 - 2.0 * w[0];
    return 3;
  }
  w[0] = 1.0;
  return 1;
}

bool merged(const sldg_ctx* c) { return (c->cfg.flags & SLDG_FLAG_MERGE_DRIFTS) != 0; }

// one step without merging: D(w/2) K(w) D(w/2) per weight
std::vector<Stage> step_stages(const sldg_ctx* c) {
  double w[3];
  const int n = strang_weights(c, w);
  std::vector<Stage> st;
  for (int i = 0; i < n; ++i) {
    st.push_back({false, false, 0.5 * w[i]});
    st.push_back({true, i == 0, w[i]});
    st.push_back({false, false, 0.5 * w[i]});
  }
  return st;
}

// merged drifts: a call of n steps is D(w_0/2), then per step the body
// K(w_0) D((w_0 + w_1)/2) ... K(w_last) D(tail), tail = (w_last + w_0)/2
// before another step of the call and w_last/2 after the last one
std::vector<Stage> merged_body(const sldg_ctx* c, bool last) {
  double w[3];
  const int n = strang_weights(c, w);
  std::vector<Stage> st;
  for (int i = 0; i < n; ++i) {
    st.push_back({true, i == 0, w[i]});
    const double next = i + 1 < n ? w[i + 1] : (last ? 0.0 : w[0]);
    st.push_back({false, false, 0.5 * (w[i] + next)});
  }
  return st;
}

// Run stages in place on buf.  FP64 storage with double-float sweeps: buf
// holds IEEE doubles where in_ieee / out_ieee say so (the call's first
// input, its last output) and double-float (hi, lo) pairs in the same
// 8-byte elements between stages, so the conversions to and from the FP32
// pipe's format happen once per call.  W of each recorded kick goes to
// Wbase[*wi] (then ++*wi), or with Wcounter to Wbase[*Wcounter] (a device
// counter the energy kernel advances; graph capture).
int run_stages(sldg_ctx* c, void* buf, const std::vector<Stage>& st, bool in_ieee, bool out_ieee,
               double* Wbase, int* Wcounter, int* wi) {
  const bool df = df_states(c);
  const int n = (int)st.size();
  for (int q = 0; q < n; ++q) {
    const bool in_df = df && (q > 0 || !in_ieee);
    const bool out_df = df && (q + 1 < n || !out_ieee);
    if (!st[q].kick) {
      SLDG_TRY(drift(c, buf, st[q].frac, in_df, out_df));
      continue;
    }
    SLDG_TRY(compute_fields(c, buf, in_df));
    if (st[q].W && Wbase) {
      KTimer t(c, SLDG_K_OTHER);
      double* slot = Wcounter ? Wbase : Wbase + *wi;
      SLDG_CU(launch_energy(c->d_E[0], c->d_E[1], c->d_wx, c->g.Dx, slot, c->stream, Wcounter));
    }
    if (st[q].W) ++*wi;
    SLDG_TRY(run_sweep(c, buf, 2, st[q].frac, false, nullptr, nullptr, in_df, df));
    SLDG_TRY(run_sweep(c, buf, 3, st[q].frac, false, nullptr, nullptr, df, out_df));
  }
  return SLDG_OK;
}

// One step (order 2 or 4, drifts not merged) in place on buf, IEEE in and
// out; W of its (first) kick field to Wslot (device) if given.
int do_step(sldg_ctx* c, void* buf, double* Wslot, int* Wcounter = nullptr) {
  int wi = 0;
  return run_stages(c, buf, step_stages(c), true, true, Wslot, Wcounter, &wi);
}

// The x-matrices of every drift fraction a step of this context uses.
int prepare_xmats(sldg_ctx* c) {
  std::vector<Stage> all = step_stages(c);
  if (merged(c)) {
    for (bool last : {false, true}) {
      std::vector<Stage> b = merged_body(c, last);
      all.insert(all.end(), b.begin(), b.end());
    }
  }
  MatSet* m;
  for (const Stage& q : all)
    if (!q.kick)
      for (int d = 0; d < 2; ++d) SLDG_TRY(ensure_xmats(c, d, q.frac, false, &m));
  return SLDG_OK;
}

// Step m of the forward again from its state src (not modified; IEEE
// doubles, or double-float pairs when src_df: the states between the steps
// of a recorded segment), keeping what the adjoint of the step needs: g2
// (the input of V1, after the x half drifts) and g3 (the input of V2, after
// V1) in the format of the step's intermediate states (double-float pairs
// when the sweeps run in double-float arithmetic), and the kick field
// (E_out, 2 D_0 D_1 doubles, nullable; the context's field holds it as
// well).  Every sweep writes out of place into the next buffer, so nothing
// is copied, and the states are those of do_step bit for bit (the same
// kernels, arithmetic and formats as the recording, which keeps double-float
// pairs between the steps of a segment).  full: finish the step into dst
// (which may be src; its previous contents are overwritten), as double-float
// pairs on FP64 storage with double-float sweeps.
int forward_stage(sldg_ctx* c, const void* src, void* g2_out, void* g3_out, double* E_out,
                  bool full, void* dst, bool src_df) {
  const bool df = df_states(c);
  SLDG_TRY(drift(c, const_cast<void*>(src), 0.5, df && src_df, df, g2_out));
  SLDG_TRY(compute_fields(c, g2_out, df));
  if (E_out) {
    SLDG_CU(cudaMemcpyAsync(E_out, c->d_E[0], c->g.Dx * sizeof(double), cudaMemcpyDeviceToDevice,
                            c->stream));
    SLDG_CU(cudaMemcpyAsync(E_out + c->g.Dx, c->d_E[1], c->g.Dx * sizeof(double),
                            cudaMemcpyDeviceToDevice, c->stream));
  }
  SLDG_TRY(run_sweep(c, g2_out, 2, 1.0, false, nullptr, nullptr, df, df, g3_out));
  if (!full) return SLDG_OK;
  SLDG_TRY(run_sweep(c, g3_out, 3, 1.0, false, nullptr, nullptr, df, df, dst));
  return drift(c, dst, 0.5, df, df);
}

// The repeated unit of sldg_step: a whole step (IEEE in and out), or with
// merged drifts the body of a step that another step follows (double-float
// pairs in and out on FP64 storage).
int run_unit(sldg_ctx* c, void* buf, double* Wslot, int* Wcounter, bool chained) {
  int wi = 0;
  if (merged(c)) return run_stages(c, buf, merged_body(c, false), false, false, Wslot, Wcounter, &wi);
  // chained: a step between two steps of the same call, whose state stays
  // in double-float pairs on FP64 storage
  return run_stages(c, buf, step_stages(c), !chained, !chained, Wslot, Wcounter, &wi);
}

// nsteps units of f as replays of one recorded unit (a CUDA graph), W of
// each to Wbase[counter++] (nullable; the device counter restarts at 0 when
// reset_counter).  *replayed stays false when graphs do not apply (fewer
// than two units, per-kernel timing on, or an earlier capture failed) and
// the caller runs the units eagerly.
int replay_steps(sldg_ctx* c, int nsteps, double* Wbase, bool reset_counter, bool* replayed,
                 bool chained = false) {
  const int hv = Wbase ? 1 : 0;
  const int k = hv + (chained ? 2 : 0);  // graph slot: unit kind, W history or not
  *replayed = false;
  if (nsteps >= 2 && !c->timing && !c->graphs_off) {
    // one recorded step replayed nsteps times: the launch overhead of the
    // small kernels goes away on small grids
    // everything the step allocates lazily exists before the capture
    SLDG_TRY(prepare_xmats(c));
    for (int d = 0; d < 2; ++d) SLDG_TRY(alloc_matset(c, &c->vm[d], c->g.Dx, false, false));
    if (!c->d_counter) SLDG_TRY(dalloc(&c->d_counter, sizeof(int)));
    if (c->step_graph[k] && (c->step_graph_buf[k] != c->f || c->step_graph_W[k] != Wbase)) {
      cudaGraphExecDestroy(c->step_graph[k]);
      c->step_graph[k] = nullptr;
    }
    if (!c->step_graph[k]) {
      const long long l0 = c->launches;
      cudaGraph_t graph = nullptr;
      bool ok = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
      const int rc = ok ? run_unit(c, c->f, Wbase, hv ? c->d_counter : nullptr, chained) : SLDG_ERR_CUDA;
      if (ok) ok = cudaStreamEndCapture(c->stream, &graph) == cudaSuccess && rc == SLDG_OK;
      if (ok) ok = cudaGraphInstantiate(&c->step_graph[k], graph, 0) == cudaSuccess;
      if (graph) cudaGraphDestroy(graph);
      c->step_graph_launches[k] = c->launches - l0;
      c->launches = l0;
      if (!ok) {
        cudaGetLastError();
        if (c->step_graph[k]) cudaGraphExecDestroy(c->step_graph[k]);
        c->step_graph[k] = nullptr;
        c->graphs_off = true;
        invalidate_vmats(c);
        c->have_field = false;
      } else {
        c->step_graph_buf[k] = c->f;
        c->step_graph_W[k] = Wbase;
      }
    }
    if (c->step_graph[k]) {
      if (hv && reset_counter) SLDG_CU(cudaMemsetAsync(c->d_counter, 0, sizeof(int), c->stream));
      for (int m = 0; m < nsteps; ++m) {
        SLDG_CU(cudaGraphLaunch(c->step_graph[k], c->stream));
        c->launches += c->step_graph_launches[k];
        c->t += c->g.dt;
        c->step += 1;
      }
      // the context's field and v-matrices belong to the last replayed step
      c->have_field = true;
      invalidate_vmats(c);
      *replayed = true;
    }
  }
  return SLDG_OK;
}

int ensure_W(sldg_ctx* c, int n) {
  if (c->W_cap >= n) return SLDG_OK;
  dfree(c->d_W);
  int cap = std::max(n, 64);
  SLDG_TRY(dalloc(&c->d_W, (size_t)cap * sizeof(double)));
  c->W_cap = cap;
  return SLDG_OK;
}

int build_tables(sldg_ctx* c) {
  const Grid& g = c->g;
  // node coordinates and weights
  std::vector<double> zall, wall[4];
  long long off[4] = {0, g.D[0], g.D[0] + g.D[1], g.D[0] + g.D[1] + g.D[2]};
  zall.resize(g.D[0] + g.D[1] + g.D[2] + g.D[3]);
  for (int d = 0; d < 4; ++d) {
    wall[d].resize(g.D[d]);
    for (long long i = 0; i < g.D[d]; ++i) {
      zall[off[d] + i] = node_coord(c, d, i);
      wall[d][i] = node_weight(c, d, i);
    }
  }
  SLDG_TRY(dalloc(&c->d_z[0], zall.size() * sizeof(double)));
  for (int d = 1; d < 4; ++d) c->d_z[d] = c->d_z[0] + off[d];
  SLDG_CU(cudaMemcpy(c->d_z[0], zall.data(), zall.size() * sizeof(double), cudaMemcpyHostToDevice));
  for (int d = 0; d < 4; ++d) {
    SLDG_TRY(dalloc(&c->d_w[d], g.D[d] * sizeof(double)));
    SLDG_CU(cudaMemcpy(c->d_w[d], wall[d].data(), g.D[d] * sizeof(double), cudaMemcpyHostToDevice));
  }
  std::vector<double> wv(g.Dv), wx(g.Dx);
  for (long long i3 = 0; i3 < g.D[3]; ++i3)
    for (long long i2 = 0; i2 < g.D[2]; ++i2) wv[i3 * g.D[2] + i2] = wall[2][i2] * wall[3][i3];
  for (long long i1 = 0; i1 < g.D[1]; ++i1)
    for (long long i0 = 0; i0 < g.D[0]; ++i0) wx[i1 * g.D[0] + i0] = wall[0][i0] * wall[1][i1];
  SLDG_TRY(dalloc(&c->d_wv, g.Dv * sizeof(double)));
  {
    std::vector<float2> wv2(g.Dv);
    for (long long i = 0; i < g.Dv; ++i) {
      const float h = (float)wv[i];
      wv2[i] = make_float2(h, (float)(wv[i] - (double)h));
    }
    SLDG_TRY(dalloc(&c->d_wv2, g.Dv * sizeof(float2)));
    SLDG_CU(cudaMemcpy(c->d_wv2, wv2.data(), g.Dv * sizeof(float2), cudaMemcpyHostToDevice));
  }
  SLDG_TRY(dalloc(&c->d_wx, g.Dx * sizeof(double)));
  SLDG_CU(cudaMemcpy(c->d_wv, wv.data(), g.Dv * sizeof(double), cudaMemcpyHostToDevice));
  SLDG_CU(cudaMemcpy(c->d_wx, wx.data(), g.Dx * sizeof(double), cudaMemcpyHostToDevice));

  // spectral tables
  for (int d = 0; d < 2; ++d) {
    const int nc = c->cfg.ncell[d];
    int K = (int)((g.D[d] - 1) / 2);
    if (K > nc - 1) K = nc - 1;
    if (c->cfg.poisson_kmax >= 0) K = c->cfg.poisson_kmax;
    c->K[d] = K;
    c->kap[d] = 2.0 * kPi / (c->cfg.hi[d] - c->cfg.lo[d]);
  }
  const int D0 = (int)g.D[0], D1 = (int)g.D[1];
  const int M1 = c->K[0] + 1, M2 = 2 * c->K[1] + 1;
  const double L0 = c->cfg.hi[0] - c->cfg.lo[0], L1 = c->cfg.hi[1] - c->cfg.lo[1];
  std::vector<double2> F1((size_t)D0 * M1), G1((size_t)M1 * D0), F2((size_t)M2 * D1), G2((size_t)D1 * M2);
  for (int n1 = 0; n1 < D0; ++n1)
    for (int m1 = 0; m1 < M1; ++m1) {
      const double ph = c->kap[0] * m1 * zall[off[0] + n1];
      const double wl = wall[0][n1] / L0;
      F1[(size_t)n1 * M1 + m1] = make_double2(wl * std::cos(ph), -wl * std::sin(ph));
      G1[(size_t)m1 * D0 + n1] = make_double2(std::cos(ph), std::sin(ph));
    }
  for (int mi = 0; mi < M2; ++mi)
    for (int n2 = 0; n2 < D1; ++n2) {
      const double ph = c->kap[1] * (mi - c->K[1]) * zall[off[1] + n2];
      const double wl = wall[1][n2] / L1;
      F2[(size_t)mi * D1 + n2] = make_double2(wl * std::cos(ph), -wl * std::sin(ph));
      G2[(size_t)n2 * M2 + mi] = make_double2(std::cos(ph), std::sin(ph));
    }
  SLDG_TRY(dalloc(&c->d_F1, F1.size() * sizeof(double2)));
  SLDG_TRY(dalloc(&c->d_G1, G1.size() * sizeof(double2)));
  SLDG_TRY(dalloc(&c->d_F2, F2.size() * sizeof(double2)));
  SLDG_TRY(dalloc(&c->d_G2, G2.size() * sizeof(double2)));
  SLDG_CU(cudaMemcpy(c->d_F1, F1.data(), F1.size() * sizeof(double2), cudaMemcpyHostToDevice));
  SLDG_CU(cudaMemcpy(c->d_G1, G1.data(), G1.size() * sizeof(double2), cudaMemcpyHostToDevice));
  SLDG_CU(cudaMemcpy(c->d_F2, F2.data(), F2.size() * sizeof(double2), cudaMemcpyHostToDevice));
  SLDG_CU(cudaMemcpy(c->d_G2, G2.data(), G2.size() * sizeof(double2), cudaMemcpyHostToDevice));
  SLDG_TRY(dalloc(&c->d_T, (size_t)D1 * M1 * sizeof(double2)));
  SLDG_TRY(dalloc(&c->d_R, 2 * (size_t)M2 * M1 * sizeof(double2)));  // c_1 rho_hat, c_2 rho_hat
  SLDG_TRY(dalloc(&c->d_U, 2 * (size_t)D1 * M1 * sizeof(double2)));
  return SLDG_OK;
}

}  // namespace

// =============================================================================
// C ABI
// =============================================================================
// The checks of sldg_init (every entry point that takes a configuration).
int sldg::validate_config(const sldg_config* cfg) {
  if (cfg->degree < 0 || cfg->degree > 3) return SLDG_ERR_BAD_CONFIG;
  for (int d = 0; d < 4; ++d) {
    if (cfg->ncell[d] < 2) return SLDG_ERR_BAD_CONFIG;
    if (!(cfg->hi[d] > cfg->lo[d]) || !std::isfinite(cfg->hi[d]) || !std::isfinite(cfg->lo[d]))
      return SLDG_ERR_BAD_CONFIG;
  }
  if (!(cfg->dt > 0.0) || !std::isfinite(cfg->dt)) return SLDG_ERR_BAD_CONFIG;
  if (cfg->precision != SLDG_FP64 && cfg->precision != SLDG_FP32) return SLDG_ERR_BAD_CONFIG;
  if (cfg->vbc != SLDG_VBC_ZERO_INFLOW && cfg->vbc != SLDG_VBC_PERIODIC) return SLDG_ERR_BAD_CONFIG;
  if (cfg->flags & ~(SLDG_FLAG_NATIVE_FP64 | SLDG_FLAG_NO_XFUSION | SLDG_FLAG_ORDER4 |
                     SLDG_FLAG_MERGE_DRIFTS | SLDG_FLAG_SPLINE))
    return SLDG_ERR_BAD_CONFIG;
  if (cfg->flags & SLDG_FLAG_SPLINE) {
    // a spline sweep stages two [n][33] tiles of a line direction on chip
    const long long esize = cfg->precision == SLDG_FP64 ? 8 : 4;
    if (cfg->degree != 0 || cfg->vbc != SLDG_VBC_PERIODIC) return SLDG_ERR_BAD_CONFIG;
    for (int d = 0; d < 4; ++d)
      if (cfg->ncell[d] < 3 || 2LL * cfg->ncell[d] * 33 * esize > 227 * 1024)
        return SLDG_ERR_BAD_CONFIG;
  }
  return SLDG_OK;
}

extern "C" {

const char* sldg_strerror(int code) {
  switch (code) {
    case SLDG_OK: return "ok";
    case SLDG_ERR_BAD_CONFIG: return "invalid or unsupported configuration";
    case SLDG_ERR_BAD_PTR: return "null or misaligned pointer";
    case SLDG_ERR_OOM: return "out of memory";
    case SLDG_ERR_CUDA: return "CUDA runtime error";
    case SLDG_ERR_NONFINITE: return "non-finite value in f";
    case SLDG_ERR_UNSUPPORTED: return "size or mode not supported";
    case SLDG_ERR_STATE: return "call out of order";
    case SLDG_ERR_ARG: return "invalid argument";
    default: return "unknown status";
  }
}

int sldg_abi_version(void) { return 2; }

int sldg_init(const sldg_config* cfg, void* f_dev, void* stream, sldg_ctx** out) {
  if (!cfg || !out) return SLDG_ERR_BAD_PTR;
  *out = nullptr;
  int rc = validate_config(cfg);
  if (rc != SLDG_OK) return rc;
  if (!f_dev || (reinterpret_cast<uintptr_t>(f_dev) & 15)) return SLDG_ERR_BAD_PTR;
  sldg_ctx* c = new (std::nothrow) sldg_ctx();
  if (!c) return SLDG_ERR_OOM;
  c->cfg = *cfg;
  c->prec = cfg->precision;
  c->esize = cfg->precision == SLDG_FP64 ? sizeof(double) : sizeof(float);
  c->f = f_dev;
  c->stream = reinterpret_cast<cudaStream_t>(stream);
  make_basis(cfg->degree + 1, &c->basis);
  Grid& g = c->g;
  g.n = cfg->degree + 1;
  for (int d = 0; d < 4; ++d) {
    g.nc[d] = cfg->ncell[d];
    g.D[d] = (long long)cfg->ncell[d] * g.n;
    g.lo[d] = cfg->lo[d];
    g.h[d] = (cfg->hi[d] - cfg->lo[d]) / cfg->ncell[d];
  }
  g.dt = cfg->dt;
  g.vbc = cfg->vbc;
  g.Dx = g.D[0] * g.D[1];
  g.Dv = g.D[2] * g.D[3];
  g.N = g.Dx * g.Dv;
  // on-chip staging limits: a whole line (x1) or a 32-column tile (x2, v1, v2)
  if (sweep_smem_bytes(c->prec, 0, g.D[0], 1) > kMaxSmem) rc = SLDG_ERR_BAD_CONFIG;
  for (int d = 1; d < 4; ++d)
    if (sweep_smem_bytes(c->prec, d, g.D[d], 1) > kMaxSmem) rc = SLDG_ERR_BAD_CONFIG;
  if (g.D[0] > 2048 || g.D[1] > 65535 || g.Dx > (1LL << 31)) rc = SLDG_ERR_BAD_CONFIG;
  for (int d = 0; d < 2; ++d)  // modes beyond (D-1)/2 are not resolved by D nodes
    if (cfg->poisson_kmax > (g.D[d] - 1) / 2) rc = SLDG_ERR_BAD_CONFIG;
  if (rc == SLDG_OK) rc = build_tables(c);
  if (rc == SLDG_OK) {
    for (int d = 0; d < 2; ++d) rc = rc ? rc : dalloc(&c->d_E[d], g.Dx * sizeof(double));
  }
  if (rc == SLDG_OK) rc = dalloc(&c->d_rho, g.Dx * sizeof(double));
  if (rc == SLDG_OK) {
    // rho partial rows: enough blocks to fill the GPU, at least 64 v-planes each
    long long ch = std::max<long long>(1, std::min<long long>(32, g.Dv / 64));
    c->rho_chunks = (int)ch;
    const size_t tabn = (size_t)(g.D[0] + g.D[1] + g.D[2] + g.D[3]);
    c->part_elems = std::max<size_t>((size_t)ch * g.Dx, diag_scratch_doubles() + tabn + 2);
    rc = dalloc(&c->d_part, c->part_elems * sizeof(double));
  }
  if (rc == SLDG_OK) rc = dalloc(&c->d_diag, 16 * sizeof(double));
  if (rc == SLDG_OK) rc = ensure_W(c, 64);
  if (rc == SLDG_OK) {
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) rc = SLDG_ERR_CUDA;
  }
  if (rc != SLDG_OK) {
    free_all(c);
    delete c;
    return rc;
  }
  *out = c;
  return SLDG_OK;
}

void sldg_destroy(sldg_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  free_all(c);
  delete c;
}

long long sldg_numel(const sldg_ctx* c) { return c ? c->g.N : 0; }

int sldg_bind(sldg_ctx* c, void* f_dev) {
  if (!c || !f_dev || (reinterpret_cast<uintptr_t>(f_dev) & 15)) return SLDG_ERR_BAD_PTR;
  c->f = f_dev;
  return SLDG_OK;
}

int sldg_set_initial(sldg_ctx* c, int kind, const double* params, int nparams) {
  if (!c) return SLDG_ERR_BAD_PTR;
  if (!params) return SLDG_ERR_BAD_PTR;
  if (kind < 0 || kind > 2 || nparams < 3) return SLDG_ERR_ARG;
  double* tab = c->d_part;  // D0+D1+D2+D3 doubles of scratch
  if (c->part_elems < (size_t)(c->g.D[0] + c->g.D[1] + c->g.D[2] + c->g.D[3])) return SLDG_ERR_UNSUPPORTED;
  int nl = 0;
  KTimer t(c, SLDG_K_OTHER, 2);
  SLDG_CU(launch_init(c->prec, c->f, c->g, kind, params, c->d_z[0], tab, c->stream, &nl));
  c->t = 0.0;
  c->step = 0;
  c->have_field = false;
  invalidate_vmats(c);
  return SLDG_OK;
}

int sldg_get_f(sldg_ctx* c, void* dst, int on_device) {
  if (!c || !dst) return SLDG_ERR_BAD_PTR;
  SLDG_CU(cudaMemcpyAsync(dst, c->f, c->g.N * c->esize,
                          on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
  if (!on_device) SLDG_CU(cudaStreamSynchronize(c->stream));
  return SLDG_OK;
}

int sldg_set_f(sldg_ctx* c, const void* src, int on_device, double t, long long step) {
  if (!c || !src) return SLDG_ERR_BAD_PTR;
  SLDG_CU(cudaMemcpyAsync(c->f, src, c->g.N * c->esize,
                          on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
  c->t = t;
  c->step = step;
  c->have_field = false;
  invalidate_vmats(c);
  return SLDG_OK;
}

int sldg_step(sldg_ctx* c, int nsteps, double* W_history) {
  if (!c) return SLDG_ERR_BAD_PTR;
  if (nsteps < 0) return SLDG_ERR_ARG;
  if (W_history) SLDG_TRY(ensure_W(c, nsteps));
  double* Wd = W_history ? c->d_W : nullptr;
  // merged drifts: D(w_0/2), nsteps - 1 bodies (replayed), the last body.
  // Double-float sweeps on FP64 storage: the first step takes IEEE doubles
  // and leaves double-float pairs, the steps between keep the pairs
  // (replayed), the last one writes IEEE doubles again, so the state is
  // converted once per call instead of twice per step.
  const bool mg = merged(c) && nsteps > 0;
  const bool dc = !mg && df_states(c) && nsteps >= 2;
  const int units = mg ? nsteps - 1 : (dc ? nsteps - 2 : nsteps);
  if (mg) {
    double w[3];
    strang_weights(c, w);
    int wi = 0;
    SLDG_TRY(run_stages(c, c->f, {{false, false, 0.5 * w[0]}}, true, false, nullptr, nullptr, &wi));
  }
  if (dc) {
    int wi = 0;
    SLDG_TRY(run_stages(c, c->f, step_stages(c), true, false, Wd, nullptr, &wi));
    c->t += c->g.dt;
    c->step += 1;
  }
  double* Wu = Wd && dc ? Wd + 1 : Wd;  // W slots of the replayed units
  bool replayed = false;
  SLDG_TRY(replay_steps(c, units, Wu, true, &replayed, dc));
  if (!replayed)
    for (int m = 0; m < units; ++m) {
      SLDG_TRY(run_unit(c, c->f, Wu ? Wu + m : nullptr, nullptr, dc));
      c->t += c->g.dt;
      c->step += 1;
    }
  if (dc) {
    int wi = 0;
    SLDG_TRY(run_stages(c, c->f, step_stages(c), false, true, Wd ? Wd + nsteps - 1 : nullptr,
                        nullptr, &wi));
    c->t += c->g.dt;
    c->step += 1;
  }
  if (mg) {
    int wi = 0;
    SLDG_TRY(run_stages(c, c->f, merged_body(c, true), false, true, Wd ? Wd + units : nullptr,
                        nullptr, &wi));
    c->t += c->g.dt;
    c->step += 1;
  }
  if (W_history && nsteps > 0) {
    SLDG_CU(cudaMemcpyAsync(W_history, c->d_W, nsteps * sizeof(double), cudaMemcpyDeviceToHost,
                            c->stream));
    SLDG_CU(cudaStreamSynchronize(c->stream));
  }
  return SLDG_OK;
}

// Host batches: batch b+1 is uploaded on a copy stream into the buffer that
// batch b-1 used while batch b is stepped on the context's stream; W of each
// batch goes to pinned host memory as soon as its step ends.
int sldg_step_host_batches(sldg_ctx* c, const void* host_f, long long batch_stride_bytes,
                           int nbatch, double* W_out) {
  if (!c || !host_f || !W_out) return SLDG_ERR_BAD_PTR;
  if (nbatch < 1 || batch_stride_bytes < 0) return SLDG_ERR_ARG;
  const size_t fb = c->g.N * c->esize;
  if (!c->d_alt) SLDG_TRY(dalloc(&c->d_alt, fb));
  if (!c->copy_stream) SLDG_CU(cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking));
  for (int i = 0; i < 2; ++i) {
    if (!c->ev_up[i]) SLDG_CU(cudaEventCreateWithFlags(&c->ev_up[i], cudaEventDisableTiming));
    if (!c->ev_free[i]) SLDG_CU(cudaEventCreateWithFlags(&c->ev_free[i], cudaEventDisableTiming));
  }
  if (c->h_W_cap < nbatch) {
    if (c->h_W) cudaFreeHost(c->h_W);
    c->h_W = nullptr;
    c->h_W_cap = 0;
    if (cudaHostAlloc(reinterpret_cast<void**>(&c->h_W), (size_t)nbatch * sizeof(double),
                      cudaHostAllocDefault) != cudaSuccess) {
      cudaGetLastError();
      c->h_W = nullptr;
      return SLDG_ERR_OOM;
    }
    c->h_W_cap = nbatch;
  }
  SLDG_TRY(ensure_W(c, nbatch));
  void* buf[2] = {c->f, c->d_alt};
  const char* src = static_cast<const char*>(host_f);
  // the copy stream may overwrite a buffer only after earlier work on it
  SLDG_CU(cudaEventRecord(c->ev_free[0], c->stream));
  SLDG_CU(cudaEventRecord(c->ev_free[1], c->stream));
  SLDG_CU(cudaStreamWaitEvent(c->copy_stream, c->ev_free[0], 0));
  SLDG_CU(cudaMemcpyAsync(buf[0], src, fb, cudaMemcpyHostToDevice, c->copy_stream));
  SLDG_CU(cudaEventRecord(c->ev_up[0], c->copy_stream));
  for (int b = 0; b < nbatch; ++b) {
    const int k = b & 1;
    if (b + 1 < nbatch) {
      const int k1 = k ^ 1;
      SLDG_CU(cudaStreamWaitEvent(c->copy_stream, c->ev_free[k1], 0));
      SLDG_CU(cudaMemcpyAsync(buf[k1], src + (size_t)(b + 1) * batch_stride_bytes, fb,
                              cudaMemcpyHostToDevice, c->copy_stream));
      SLDG_CU(cudaEventRecord(c->ev_up[k1], c->copy_stream));
    }
    SLDG_CU(cudaStreamWaitEvent(c->stream, c->ev_up[k], 0));
    c->have_field = false;
    invalidate_vmats(c);
    SLDG_TRY(do_step(c, buf[k], c->d_W + b));
    SLDG_CU(cudaEventRecord(c->ev_free[k], c->stream));
    SLDG_CU(cudaMemcpyAsync(c->h_W + b, c->d_W + b, sizeof(double), cudaMemcpyDeviceToHost,
                            c->stream));
  }
  if ((nbatch - 1) & 1)  // the last state sits in the second buffer
    SLDG_CU(cudaMemcpyAsync(c->f, c->d_alt, fb, cudaMemcpyDeviceToDevice, c->stream));
  SLDG_CU(cudaStreamSynchronize(c->stream));
  std::memcpy(W_out, c->h_W, (size_t)nbatch * sizeof(double));
  c->t += c->g.dt;
  c->step += 1;
  return SLDG_OK;
}

int sldg_sweep(sldg_ctx* c, int dim, double frac) {
  if (!c) return SLDG_ERR_BAD_PTR;
  if (dim < 0 || dim > 3 || !std::isfinite(frac)) return SLDG_ERR_ARG;
  return run_sweep(c, c->f, dim, frac, false, nullptr, nullptr);
}

int sldg_drift(sldg_ctx* c, double frac) {
  if (!c) return SLDG_ERR_BAD_PTR;
  if (!std::isfinite(frac)) return SLDG_ERR_ARG;
  return drift(c, c->f, frac, false, false);
}

int sldg_compute_fields(sldg_ctx* c) {
  if (!c) return SLDG_ERR_BAD_PTR;
  return compute_fields(c, c->f);
}

int sldg_set_field(sldg_ctx* c, const double* E1, const double* E2, int on_device) {
  if (!c || !E1 || !E2) return SLDG_ERR_BAD_PTR;
  const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  SLDG_CU(cudaMemcpyAsync(c->d_E[0], E1, c->g.Dx * sizeof(double), k, c->stream));
  SLDG_CU(cudaMemcpyAsync(c->d_E[1], E2, c->g.Dx * sizeof(double), k, c->stream));
  if (!on_device) SLDG_CU(cudaStreamSynchronize(c->stream));
  c->have_field = true;
  invalidate_vmats(c);
  return SLDG_OK;
}

int sldg_fields(sldg_ctx* c, double* rho, double* E1, double* E2, int on_device) {
  if (!c) return SLDG_ERR_BAD_PTR;
  const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  const size_t b = c->g.Dx * sizeof(double);
  if (rho) SLDG_CU(cudaMemcpyAsync(rho, c->d_rho, b, k, c->stream));
  if (E1) SLDG_CU(cudaMemcpyAsync(E1, c->d_E[0], b, k, c->stream));
  if (E2) SLDG_CU(cudaMemcpyAsync(E2, c->d_E[1], b, k, c->stream));
  if (!on_device) SLDG_CU(cudaStreamSynchronize(c->stream));
  return SLDG_OK;
}

int sldg_diagnostics(sldg_ctx* c, sldg_diag* out) {
  if (!c || !out) return SLDG_ERR_BAD_PTR;
  SLDG_TRY(compute_fields(c, c->f));
  int nl = 0;
  {
    KTimer t(c, SLDG_K_OTHER, 3);
    SLDG_CU(launch_diag(c->prec, c->f, c->g, c->d_wx, c->d_wv, c->d_z[2], c->d_z[3], c->d_part,
                        c->d_diag, c->stream, &nl));
    SLDG_CU(launch_energy(c->d_E[0], c->d_E[1], c->d_wx, c->g.Dx, c->d_diag + 4, c->stream));
  }
  double h[5];
  SLDG_CU(cudaMemcpyAsync(h, c->d_diag, 5 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  SLDG_CU(cudaStreamSynchronize(c->stream));
  out->t = c->t;
  out->step = c->step;
  out->mass = h[0];
  out->l1 = h[1];
  out->l2sq = h[2];
  out->kinetic = h[3];
  out->electric = h[4];
  out->total = h[3] + h[4];
  for (int i = 0; i < 5; ++i)
    if (!std::isfinite(h[i])) return SLDG_ERR_NONFINITE;
  return SLDG_OK;
}

// ---- adjoint ------------------------------------------------------------------------
// The backward's state-sized working memory: the recomputation slots, the
// intermediates of an adjoint step and the recomputed kick fields
static void release_backward_scratch(sldg_ctx* c) {
  dfree(c->d_seg);
  c->seg_count = 0;
  for (int i = 0; i < 2; ++i) dfree(c->d_work[i]);
  dfree(c->d_Ecap);
  c->Ecap_steps = 0;
}

static int ensure_adjoint_scratch(sldg_ctx* c) {
  const Grid& g = c->g;
  for (int d = 0; d < 2; ++d)
    if (!c->d_Eb[d]) SLDG_TRY(dalloc(&c->d_Eb[d], g.Dx * sizeof(double)));
  if (!c->d_rhob) SLDG_TRY(dalloc(&c->d_rhob, g.Dx * sizeof(double)));
  const size_t need = (size_t)std::max(g.D[2], g.D[3]) * g.Dx;
  if (c->epart_elems < need) {
    dfree(c->d_epart);
    SLDG_TRY(dalloc(&c->d_epart, need * sizeof(double)));
    c->epart_elems = need;
  }
  return SLDG_OK;
}

int sldg_sweep_adjoint(sldg_ctx* c, int dim, double frac, void* lam, const void* g, double* Ebar) {
  if (!c || !lam) return SLDG_ERR_BAD_PTR;
  if (dim < 0 || dim > 3 || !std::isfinite(frac)) return SLDG_ERR_ARG;
  if ((g == nullptr) != (Ebar == nullptr)) return SLDG_ERR_ARG;
  if (g && dim < 2) return SLDG_ERR_ARG;
  if (spline(c)) return SLDG_ERR_UNSUPPORTED;
  if (g) SLDG_TRY(ensure_adjoint_scratch(c));
  return run_sweep(c, lam, dim, frac, true, g, Ebar);
}

int sldg_record(sldg_ctx* c, int nsteps, int ckpt_every, double* W_history) {
  if (!c) return SLDG_ERR_BAD_PTR;
  if (c->cfg.flags & (SLDG_FLAG_ORDER4 | SLDG_FLAG_MERGE_DRIFTS | SLDG_FLAG_SPLINE))
    return SLDG_ERR_UNSUPPORTED;
  if (nsteps < 1 || ckpt_every < 1) return SLDG_ERR_ARG;
  const size_t fb = c->g.N * c->esize;
  const size_t nck = (nsteps + ckpt_every - 1) / ckpt_every;
  c->recorded = false;
  // the pool, the W history and the backward's working copies stay allocated
  // between recordings (the replayed step graph keeps its W buffer); a pool
  // that does not fit beside the backward's copies takes their memory
  if (c->ck_cap < nck) {
    dfree(c->d_ckpool);
    c->ck_cap = 0;
    if (dalloc(&c->d_ckpool, nck * fb) != SLDG_OK) {
      release_backward_scratch(c);
      SLDG_TRY(dalloc(&c->d_ckpool, nck * fb));
    }
    c->ck_cap = nck;
  }
  if (c->Wrec_cap < nsteps) {
    dfree(c->d_Wrec);
    c->Wrec_cap = 0;
    SLDG_TRY(dalloc(&c->d_Wrec, nsteps * sizeof(double)));
    c->Wrec_cap = nsteps;
  }
  c->ck_count = nck;
  c->rec_t0 = c->t;
  c->rec_step0 = c->step;
  for (int m0 = 0; m0 < nsteps; m0 += ckpt_every) {
    char* dst = reinterpret_cast<char*>(c->d_ckpool) + (size_t)(m0 / ckpt_every) * fb;
    SLDG_CU(cudaMemcpyAsync(dst, c->f, fb, cudaMemcpyDeviceToDevice, c->stream));
    const int ns = std::min(ckpt_every, nsteps - m0);
    // double-float sweeps: the state stays in double-float pairs between the
    // steps of a segment (IEEE at its ends, where the checkpoints are taken)
    const bool dc = df_states(c) && ns >= 2;
    int a = m0, b = m0 + ns;  // steps run as whole units
    if (dc) {
      int wi = 0;
      SLDG_TRY(run_stages(c, c->f, step_stages(c), true, false, c->d_Wrec + m0, nullptr, &wi));
      c->t += c->g.dt;
      c->step += 1;
      ++a;
      --b;
    }
    bool replayed = false;
    if (b - a >= 2 && !c->timing && !c->graphs_off) {
      if (!c->d_counter) SLDG_TRY(dalloc(&c->d_counter, sizeof(int)));
      SLDG_CU(launch_set_int(c->d_counter, a, c->stream));  // W of step a + i to d_Wrec[a + i]
      SLDG_TRY(replay_steps(c, b - a, c->d_Wrec, false, &replayed, dc));
    }
    if (!replayed)
      for (int m = a; m < b; ++m) {
        SLDG_TRY(run_unit(c, c->f, c->d_Wrec + m, nullptr, dc));
        c->t += c->g.dt;
        c->step += 1;
      }
    if (dc) {
      int wi = 0;
      SLDG_TRY(run_stages(c, c->f, step_stages(c), false, true, c->d_Wrec + b, nullptr, &wi));
      c->t += c->g.dt;
      c->step += 1;
    }
  }
  if (W_history) {
    SLDG_CU(cudaMemcpyAsync(W_history, c->d_Wrec, nsteps * sizeof(double), cudaMemcpyDeviceToHost,
                            c->stream));
    SLDG_CU(cudaStreamSynchronize(c->stream));
  }
  c->rec_nsteps = nsteps;
  c->rec_ckpt = ckpt_every;
  c->recorded = true;
  return SLDG_OK;
}

int sldg_set_slot_limit(sldg_ctx* c, int max_slots) {
  if (!c) return SLDG_ERR_BAD_PTR;
  if (max_slots < 0) return SLDG_ERR_ARG;
  c->slot_limit = max_slots;
  return SLDG_OK;
}

int sldg_backward_stats(const sldg_ctx* c, long long* recomputed_steps, int* slots) {
  if (!c) return SLDG_ERR_BAD_PTR;
  if (recomputed_steps) *recomputed_steps = c->bwd_recomputed;
  if (slots) *slots = (int)c->seg_count;
  return SLDG_OK;
}

}  // extern "C"

namespace {

// The backward keeps the adjoint in double-float pairs on FP64 storage with
// double-float sweeps (no conversion through the FP64 pipe in its passes);
// sldg_backward converts the gradient to IEEE doubles at the end.
bool lam_df(const sldg_ctx* c) { return df_states(c); }

// Adjoint of a half drift X2(tau/2) X1(tau/2) on the adjoint in place: one
// fused pass of the transposed sweeps, or X2^T then X1^T.  rho_fold: first
// the charge-density adjoint lam += w_v rho_bar(x) (the adjoint of the
// density the drift's output fed), inside the fused pass's staging or as
// its own kernel (on IEEE doubles)
int adjoint_drift(sldg_ctx* c, void* lam, bool rho_fold = false) {
  const bool ldf = lam_df(c);
  bool fused = false;
  SLDG_TRY(run_x12(c, lam, 0.5, ldf, ldf, &fused, true, nullptr, rho_fold));
  if (!fused) {
    bool in_df = ldf;
    if (rho_fold) {
      if (in_df) {
        KTimer t(c, SLDG_K_OTHER);
        SLDG_CU(launch_df_to_ieee(lam, lam, c->g.N, c->stream));
        in_df = false;
      }
      KTimer t(c, SLDG_K_RHO);
      SLDG_CU(launch_rho_adj(c->prec, lam, c->g, c->d_wv, c->d_rhob, c->stream));
    }
    SLDG_TRY(run_sweep(c, lam, 1, 0.5, true, nullptr, nullptr, in_df, ldf));
    SLDG_TRY(run_sweep(c, lam, 0, 0.5, true, nullptr, nullptr, ldf, ldf));
  }
  return SLDG_OK;
}

// Adjoint of Strang step m (global index) from its forward intermediates g2
// (input of V1) and g3 (input of V2) and its kick field (E: 2 D_0 D_1
// doubles, or null when the context's field is already the step's):
// grad <- (step m)^T grad + the dJ/dW_m c_m contributions (Eq. AB-sldg
// transposed, the v-shift derivatives, the Poisson and charge-density
// adjoints).
int adjoint_step_from(sldg_ctx* c, const void* g2, const void* g3, const double* E, int m,
                      const double* cW, void* grad) {
  const Grid& g = c->g;
  if (E) {
    SLDG_CU(cudaMemcpyAsync(c->d_E[0], E, g.Dx * sizeof(double), cudaMemcpyDeviceToDevice,
                            c->stream));
    SLDG_CU(cudaMemcpyAsync(c->d_E[1], E + g.Dx, g.Dx * sizeof(double), cudaMemcpyDeviceToDevice,
                            c->stream));
    c->have_field = true;
    invalidate_vmats(c);
  }
  SLDG_CU(cudaMemsetAsync(c->d_Eb[0], 0, g.Dx * sizeof(double), c->stream));
  SLDG_CU(cudaMemsetAsync(c->d_Eb[1], 0, g.Dx * sizeof(double), c->stream));
  SLDG_TRY(adjoint_drift(c, grad));
  const bool gdf = df_states(c);  // g2, g3 as forward_stage keeps them
  const bool ldf = lam_df(c);
  SLDG_TRY(run_sweep(c, grad, 3, 1.0, true, g3, c->d_Eb[1], ldf, ldf, nullptr, gdf));
  SLDG_TRY(run_sweep(c, grad, 2, 1.0, true, g2, c->d_Eb[0], ldf, ldf, nullptr, gdf));
  {
    KTimer t(c, SLDG_K_OTHER);
    SLDG_CU(launch_energy_adj(c->d_Eb[0], c->d_Eb[1], c->d_E[0], c->d_E[1], c->d_wx, g.Dx,
                              cW ? cW[m] : g.dt, c->stream));
  }
  {
    int nl = 0;
    KTimer t(c, SLDG_K_POISSON, 4);
    SLDG_CU(launch_poisson_adj(poisson_args(c), c->d_Eb[0], c->d_Eb[1], c->d_rhob, c->stream, &nl));
  }
  return adjoint_drift(c, grad, true);
}

// The same from the step's initial state fm (recomputing g2, g3 and the
// field in the two work buffers)
int adjoint_step(sldg_ctx* c, const void* fm, int m, const double* cW, void* grad, bool fm_df) {
  void* g2 = c->d_work[0];
  void* g3 = c->d_work[1];
  SLDG_TRY(forward_stage(c, fm, g2, g3, nullptr, false, nullptr, fm_df));
  return adjoint_step_from(c, g2, g3, nullptr, m, cW, grad);
}

// dst <- src advanced by k Strang steps
// dst <- src advanced by k >= 1 Strang steps inside a recorded segment: src
// in IEEE doubles or (src_df) double-float pairs, dst as double-float pairs
// on FP64 storage with double-float sweeps (the recording's states there)
int advance(sldg_ctx* c, void* dst, const void* src, int k, bool src_df) {
  const size_t fb = c->g.N * c->esize;
  if (dst != src) SLDG_CU(cudaMemcpyAsync(dst, src, fb, cudaMemcpyDeviceToDevice, c->stream));
  for (int i = 0; i < k; ++i) {
    int wi = 0;
    SLDG_TRY(run_stages(c, dst, step_stages(c), i == 0 && !src_df, false, nullptr, nullptr, &wi));
  }
  c->bwd_recomputed += k;
  return SLDG_OK;
}

// Adjoint of steps [a, b), src holding the state at step a (not modified),
// with the recomputation slots in `free` (at least one).  As many states as
// slots allow are stored and consumed in reverse; otherwise the range is
// split at its midpoint (the state there goes to one slot) and the halves are
// treated later half first; with a single slot every state is recomputed from
// src.  Recomputation: none beyond one pass when b - a - 1 <= slots, about
// log2(b - a) passes when slots run out.
int adjoint_range(sldg_ctx* c, const void* src, int a, int b, std::vector<char*>& free,
                  const double* cW, void* grad, bool src_df) {
  const size_t fb = c->g.N * c->esize;
  const int n = b - a;
  if (n == 1) return adjoint_step(c, src, a, cW, grad, src_df);
  if ((size_t)(2 * n + 1) <= free.size() && c->d_Ecap && n <= c->Ecap_steps) {
    // one forward pass over the range keeps every step's g2, g3 and field
    std::vector<char*> st(free.end() - (2 * n + 1), free.end());
    free.resize(free.size() - (2 * n + 1));
    char* w = st[2 * n];  // the running state from step a + 1 on (src is kept)
    const long long e2 = 2 * c->g.Dx;
    for (int i = 0; i < n; ++i) {
      SLDG_TRY(forward_stage(c, i == 0 ? src : w, st[2 * i], st[2 * i + 1], c->d_Ecap + i * e2,
                             i + 1 < n, w, i == 0 ? src_df : true));
      if (i + 1 < n) c->bwd_recomputed += 1;
    }
    for (int m = b - 1; m >= a; --m)
      SLDG_TRY(adjoint_step_from(c, st[2 * (m - a)], st[2 * (m - a) + 1],
                                 c->d_Ecap + (m - a) * e2, m, cW, grad));
    free.insert(free.end(), st.begin(), st.end());
    return SLDG_OK;
  }
  if ((size_t)(n - 1) <= free.size()) {  // store states a+1 .. b-1, then walk back
    std::vector<char*> st(free.end() - (n - 1), free.end());
    free.resize(free.size() - (n - 1));
    const void* prev = src;
    for (int i = 0; i < n - 1; ++i) {
      SLDG_TRY(advance(c, st[i], prev, 1, i == 0 ? src_df : true));
      prev = st[i];
    }
    for (int m = b - 1; m > a; --m) SLDG_TRY(adjoint_step(c, st[m - a - 1], m, cW, grad, true));
    SLDG_TRY(adjoint_step(c, src, a, cW, grad, src_df));
    free.insert(free.end(), st.begin(), st.end());
    return SLDG_OK;
  }
  if (free.size() == 1) {  // one slot: recompute every state from src
    char* w = free.back();
    for (int m = b - 1; m > a; --m) {
      SLDG_TRY(advance(c, w, src, m - a, src_df));
      SLDG_TRY(adjoint_step(c, w, m, cW, grad, true));
    }
    return adjoint_step(c, src, a, cW, grad, src_df);
  }
  const int mid = a + n / 2;
  char* s = free.back();
  free.pop_back();
  SLDG_TRY(advance(c, s, src, mid - a, src_df));
  SLDG_TRY(adjoint_range(c, s, mid, b, free, cW, grad, true));
  free.push_back(s);
  (void)fb;
  return adjoint_range(c, src, a, mid, free, cW, grad, src_df);
}

}  // namespace

extern "C" {

// J = sum_m c_m W_m of the last recording, c_m = cW[m] or dt: a compensated
// (Neumaier) sum on the host of the recorded W history
static int recorded_objective(sldg_ctx* c, const double* cW, double* J) {
  const int n = c->rec_nsteps;
  std::vector<double> W(n);
  SLDG_CU(cudaMemcpyAsync(W.data(), c->d_Wrec, n * sizeof(double), cudaMemcpyDeviceToHost,
                          c->stream));
  SLDG_CU(cudaStreamSynchronize(c->stream));
  double s = 0.0, comp = 0.0;
  for (int m = 0; m < n; ++m) {
    const double x = (cW ? cW[m] : c->g.dt) * W[m];
    const double t = s + x;
    comp += std::fabs(s) >= std::fabs(x) ? (s - t) + x : (x - t) + s;
    s = t;
  }
  *J = s + comp;
  return SLDG_OK;
}

int sldg_objective(sldg_ctx* c, const double* cW, int ncW, double* J_out) {
  if (!c || !J_out) return SLDG_ERR_BAD_PTR;
  if (!c->recorded) return SLDG_ERR_STATE;
  if (cW && ncW != c->rec_nsteps) return SLDG_ERR_ARG;
  return recorded_objective(c, cW, J_out);
}

int sldg_backward(sldg_ctx* c, const double* cW, int ncW, void* grad, double* J_out) {
  if (!c || !grad) return SLDG_ERR_BAD_PTR;
  if (c->cfg.flags & (SLDG_FLAG_ORDER4 | SLDG_FLAG_MERGE_DRIFTS | SLDG_FLAG_SPLINE))
    return SLDG_ERR_UNSUPPORTED;
  if (!c->recorded) return SLDG_ERR_STATE;
  if (cW && ncW != c->rec_nsteps) return SLDG_ERR_ARG;
  const Grid& g = c->g;
  const int n = c->rec_nsteps, ck = c->rec_ckpt;
  const size_t fb = g.N * c->esize;
  char* pool = reinterpret_cast<char*>(c->d_ckpool);
  if (J_out) SLDG_TRY(recorded_objective(c, cW, J_out));
  // working memory: g2, g3 and the recomputation slots (as many as a segment
  // can use, within the free device memory and the slot limit)
  for (int i = 0; i < 2; ++i)
    if (!c->d_work[i]) SLDG_TRY(dalloc(&c->d_work[i], fb));
  SLDG_TRY(ensure_adjoint_scratch(c));
  // as many slots as a segment can use: 2 S + 1 keep every step's g2, g3
  const size_t want = (size_t)(2 * std::min(ck, n) + 1);
  if (!c->d_Ecap || c->Ecap_steps < std::min(ck, n)) {
    dfree(c->d_Ecap);
    c->Ecap_steps = 0;
    SLDG_TRY(dalloc(&c->d_Ecap, (size_t)std::min(ck, n) * 2 * g.Dx * sizeof(double)));
    c->Ecap_steps = std::min(ck, n);
  }
  size_t slots = want;
  if (c->slot_limit > 0) slots = std::min(slots, (size_t)c->slot_limit);
  if (c->seg_count != slots) {
    dfree(c->d_seg);
    c->seg_count = 0;
    size_t freeb = 0, totalb = 0;
    SLDG_CU(cudaMemGetInfo(&freeb, &totalb));
    const size_t margin = std::max<size_t>(totalb / 64, (size_t)1 << 30);
    const size_t fit = freeb > margin ? (freeb - margin) / fb : 0;
    slots = std::min(slots, fit);
    if (slots < 1) return SLDG_ERR_OOM;
    SLDG_TRY(dalloc(&c->d_seg, slots * fb));
    c->seg_count = slots;
  }
  std::vector<char*> free;
  for (size_t i = 0; i < c->seg_count; ++i) free.push_back(reinterpret_cast<char*>(c->d_seg) + i * fb);
  c->bwd_recomputed = 0;
  SLDG_CU(cudaMemsetAsync(grad, 0, fb, c->stream));
  const int nseg = (int)c->ck_count;
  for (int sidx = nseg - 1; sidx >= 0; --sidx) {
    const int m0 = sidx * ck, m1 = std::min(m0 + ck, n);
    SLDG_TRY(adjoint_range(c, pool + (size_t)sidx * fb, m0, m1, free, cW, grad, false));
  }
  if (lam_df(c)) {  // the zero start reads as pairs; the result goes out as doubles
    KTimer t(c, SLDG_K_OTHER);
    SLDG_CU(launch_df_to_ieee(grad, grad, g.N, c->stream));
  }
  // the context's field now belongs to the first step; leave f as recorded
  c->have_field = false;
  invalidate_vmats(c);
  return SLDG_OK;
}

int sldg_initial_param_grad(sldg_ctx* c, int kind, const double* params, int nparams,
                            const void* grad, double* out) {
  if (!c || !params || !grad || !out) return SLDG_ERR_BAD_PTR;
  if (kind < 0 || kind > 2 || nparams < 3) return SLDG_ERR_ARG;
  const Grid& g = c->g;
  const size_t tabn = g.D[0] + g.D[1] + g.D[2] + g.D[3];
  if (c->part_elems < tabn + diag_scratch_doubles() + 2) {
    // scratch layout: [tab][partials][result]
    dfree(c->d_part);
    c->part_elems = std::max(c->part_elems, tabn + diag_scratch_doubles() + 2);
    SLDG_TRY(dalloc(&c->d_part, c->part_elems * sizeof(double)));
  }
  double* tab = c->d_part;
  double* scratch = c->d_part + tabn;
  double* res = c->d_part + tabn + diag_scratch_doubles();
  int nl = 0;
  {
    KTimer t(c, SLDG_K_OTHER, 3);
    SLDG_CU(launch_param_grad(c->prec, grad, g, kind, params, c->d_z[0], tab, scratch, res, c->stream, &nl));
  }
  SLDG_CU(cudaMemcpyAsync(out, res, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  SLDG_CU(cudaStreamSynchronize(c->stream));
  return SLDG_OK;
}

// ---- measurement ----------------------------------------------------------------------
long long sldg_launch_count(const sldg_ctx* c) { return c ? c->launches : 0; }

int sldg_x_pass_shape(const sldg_ctx* c, int* cluster_ctas, int* lanes_per_line_pair) {
  if (!c) return SLDG_ERR_BAD_PTR;
  if (cluster_ctas) *cluster_ctas = c->x12_shape[0];
  if (lanes_per_line_pair) *lanes_per_line_pair = c->x12_shape[1];
  return SLDG_OK;
}

int sldg_timing(sldg_ctx* c, int enable) {
  if (!c) return SLDG_ERR_BAD_PTR;
  SLDG_CU(cudaStreamSynchronize(c->stream));
  if (enable && c->ev_pool.empty()) {
    c->ev_pool.resize(2 * kTimerPairs);
    for (auto& e : c->ev_pool) SLDG_CU(cudaEventCreate(&e));
    c->ev_kind.assign(kTimerPairs, 0);
  }
  c->timing = enable != 0;
  c->ev_used = 0;
  for (int k = 0; k < SLDG_NUM_KINDS; ++k) {
    c->acc_ms[k] = 0.0;
    c->acc_n[k] = 0;
  }
  return SLDG_OK;
}

int sldg_timing_read(sldg_ctx* c, double* ms, long long* count) {
  if (!c) return SLDG_ERR_BAD_PTR;
  SLDG_CU(cudaStreamSynchronize(c->stream));
  for (size_t i = 0; i < c->ev_used; ++i) {
    float t = 0.f;
    SLDG_CU(cudaEventElapsedTime(&t, c->ev_pool[2 * i], c->ev_pool[2 * i + 1]));
    c->acc_ms[c->ev_kind[i]] += t;
  }
  c->ev_used = 0;
  for (int k = 0; k < SLDG_NUM_KINDS; ++k) {
    if (ms) ms[k] = c->acc_ms[k];
    if (count) count[k] = c->acc_n[k];
  }
  return SLDG_OK;
}

}  // extern "C"
