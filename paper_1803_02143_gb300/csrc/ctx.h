// ctx.h -- host-side context of libsldg and the launch interface between
// its translation units.
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "common.cuh"

namespace sldg {

// Matrices of one family of shifts, structure-of-arrays so that consecutive
// threads (consecutive keys) read consecutive addresses:
//   ab[(k * count) + key], k = 0..n*n-1 for A (row-major), n*n..2n*n-1 for B;
//   dab likewise for dA/dtheta, dB/dtheta (only when derivatives requested);
//   s[key] the integer cell shift.
struct MatSet {
  void* ab = nullptr;   // element type of the context precision
  void* dab = nullptr;  // same precision, derivative matrices
  void* ab2 = nullptr;  // FP64 contexts: (hi, lo) float pairs of ab, same layout
  int* s = nullptr;
  // transposed sweep in forward form: [B^T; A^T] applied to source cells
  // c + s and c + s + 1, i.e. shift entries -s - 1 (built on demand)
  void* dab2 = nullptr;  // FP64 contexts: (hi, lo) float pairs of dab
  void* abt = nullptr;   // context precision
  void* abt2 = nullptr;  // FP64 contexts: (hi, lo) float pairs
  int* st = nullptr;
  bool with_t = false;
  long long count = 0;
  double frac = 0.0;    // shift scale these matrices were built for
  bool valid = false;
  bool with_deriv = false;
};

// Everything a sweep launch needs.
struct SweepArgs {
  void* f;             // in place, N elements
  void* out;           // or null: outputs to out (N elements), f read only; only the
                       // strided kernels take it (launch_sweep_* return
                       // cudaErrorNotSupported for the others)
  const void* g;       // forward input for the shift derivative (adjoint v-sweeps), or null
  double* epart;       // partial sums of the shift derivative, or null
  int prec;            // SLDG_FP64 / SLDG_FP32
  int n;               // nodes per cell
  int dim;             // 0..3
  int nc;              // cells along dim
  long long inner;     // elements between consecutive nodes along dim
  long long outer;     // number of (D x inner) blocks
  const void* ab;      // matrices (SoA), see MatSet
  const void* ab2;     // the same matrices as (hi, lo) float pairs (FP64 contexts)
  const void* dab;
  const void* dab2;    // (hi, lo) pairs of dab (FP64 contexts)
  const int* s;
  long long mcount;    // keys in the matrix set
  long long key_div;   // x-sweeps: key = (line or block index / key_div) % key_mod
  long long key_mod;   // v-sweeps: key = column % key_mod
  int periodic;
  int adjoint;
  int lines_per_tile;  // x1-sweep tile height R (divides D1)
  int native_fp64;     // FP64 storage: 1 = FP64 FMA kernels, 0 = double-float kernels
  int in_df;           // double-float kernels: input elements are (hi, lo) pairs
  int out_df;          // double-float kernels: write (hi, lo) pairs instead of doubles
  int g_df;            // g holds (hi, lo) pairs instead of doubles (FP64 contexts)
  const void* tab2;    // shift-derivative kernel of FP64 contexts: with ts non-null it also
  const int* ts;       // applies the transposed sweep (pairs tab2, shifts ts) in place
};

// An out-of-place request (outputs to a buffer other than the input).
inline bool out_of_place(const SweepArgs& a) { return a.out && a.out != a.f; }

// Kernel launchers (sweep_f64.cu / sweep_f32.cu).
cudaError_t launch_sweep_f64(const SweepArgs& a, cudaStream_t st);  // FP64 FMA
cudaError_t launch_sweep_df(const SweepArgs& a, cudaStream_t st);   // double-float
// cubic-spline advection (spline.cu): a.ab holds theta per key (context
// precision), a.s the integer shifts; degree 0, periodic lines of >= 3 points
cudaError_t launch_spline_sweep(const SweepArgs& a, cudaStream_t st);
cudaError_t launch_spline_shifts(int prec, long long count, const double* src, double dt,
                                 double frac, double h, void* theta, int* s, cudaStream_t st);
// shift-derivative partials of an adjoint v-sweep in double-float (a.f = the
// adjoint before the sweep, a.g = the forward input, a.dab2, a.s, a.epart)
cudaError_t launch_ebar_df(const SweepArgs& a, cudaStream_t st);
cudaError_t launch_sweep_f32(const SweepArgs& a, cudaStream_t st);
// fused X1, X2 of FP32 storage (sweep_f32.cu); cudaErrorNotSupported if the
// layout does not fit.  shape (nullable, two ints): the launch's CTAs per
// x-plane (cluster size) and lanes per x1 line pair of its X1 phase.  out
// (nullable): write the result there and leave f unchanged.  fold_w, fold_r
// (nullable): first add fold_w[v] * fold_r[x] to every input element (the
// charge-density adjoint ahead of a transposed pass, as launch_rho_adj).
cudaError_t launch_sweep_x12_f32(void* f, const Grid& g, const void* ab1, const int* s1,
                                 const void* ab2, const int* s2, cudaStream_t st,
                                 int* shape = nullptr, void* out = nullptr,
                                 const double* fold_w = nullptr, const double* fold_r = nullptr);
// the same for FP64 storage in double-float arithmetic (sweep_df_x12.cu); ab1, ab2
// are the (hi, lo) float-pair tables, in_df / out_df the element formats (the
// fold adds to either format)
cudaError_t launch_sweep_x12_df(void* f, const Grid& g, const void* ab1, const int* s1,
                                const void* ab2, const int* s2, int in_df, int out_df,
                                cudaStream_t st, int* shape = nullptr, void* out = nullptr,
                                const double* fold_w = nullptr, const double* fold_r = nullptr);
size_t sweep_smem_bytes(int prec, int dim, long long D, int lines_per_tile);
// SLDG_OK or SLDG_ERR_BAD_CONFIG: the configuration checks of sldg_init (api.cu)
int validate_config(const sldg_config* cfg);

}  // namespace sldg

struct sldg_ctx {
  sldg_config cfg;
  sldg::Grid g;
  sldg::Basis basis;
  int prec;
  size_t esize;
  void* f;
  cudaStream_t stream;

  // per-direction node coordinates and weights (device, D_d doubles)
  double* d_z[4] = {nullptr, nullptr, nullptr, nullptr};
  double* d_w[4] = {nullptr, nullptr, nullptr, nullptr};
  double* d_wv = nullptr;  // v-plane weights w_v1 * w_v2, Dv doubles
  float2* d_wv2 = nullptr; // the same weights as (hi, lo) float pairs
  double* d_wx = nullptr;  // x-plane weights w_x1 * w_x2, Dx doubles

  // x1: key v1 node, x2: key v2 node; a few shift fractions at a time (the
  // drifts of the order-4 and merged splittings use up to three)
  static constexpr int kXSlots = 6;
  sldg::MatSet xm[2][kXSlots];
  int xm_next[2] = {0, 0};  // slot replaced next when all are taken
  sldg::MatSet vm[2];  // v1, v2: key x-node

  // fields
  double* d_rho = nullptr;
  double* d_E[2] = {nullptr, nullptr};
  bool have_field = false;

  // reduction scratch
  double* d_part = nullptr;
  size_t part_elems = 0;
  int rho_chunks = 1;

  // spectral tables (complex as double2), K = modes per direction
  int K[2] = {0, 0};
  double2* d_F1 = nullptr;  // [D0][K0+1]   w_n/L exp(-i k m z_n), m >= 0
  double2* d_F2 = nullptr;  // [2K1+1][D1]  w_n/L exp(-i k m z_n), m = -K1..K1
  double2* d_G1 = nullptr;  // [K0+1][D0]   exp(+i k m z_n)
  double2* d_G2 = nullptr;  // [D1][2K1+1]  exp(+i k m z_n)
  double2* d_T = nullptr;   // work [D1][K0+1]
  double2* d_R = nullptr;   // work [2K1+1][K0+1]
  double2* d_U = nullptr;   // work 2 x [D1][K0+1]
  double kap[2] = {0.0, 0.0};

  // per-step electric energy (device) and diagnostics scratch
  double* d_W = nullptr;
  int W_cap = 0;
  double* d_diag = nullptr;  // small result buffer

  // adjoint
  void* d_ckpool = nullptr;  // checkpoints: ck_count in use of ck_cap allocated
  size_t ck_count = 0, ck_cap = 0;
  int rec_nsteps = 0, rec_ckpt = 0;
  bool recorded = false;
  double* d_Wrec = nullptr;  // recorded W history, Wrec_cap doubles allocated
  int Wrec_cap = 0;
  void* d_work[4] = {nullptr, nullptr, nullptr, nullptr};  // g2, g3 of the adjoint step
  void* d_seg = nullptr;        // recomputation slots, seg_count states of f
  size_t seg_count = 0;
  int slot_limit = 0;           // upper bound on seg_count (0: as many as fit)
  double* d_Ecap = nullptr;     // kick fields of a recomputed segment, [steps][2][Dx]
  int Ecap_steps = 0;
  long long bwd_recomputed = 0; // Strang steps recomputed by the last backward
  double* d_Eb[2] = {nullptr, nullptr};
  double* d_rhob = nullptr;
  double* d_epart = nullptr;
  size_t epart_elems = 0;
  void* rec_f0_state = nullptr;
  double rec_t0 = 0.0;
  long long rec_step0 = 0;

  // host-batch pipeline (sldg_step_host_batches): a second state buffer, a
  // copy stream, and pinned host slots for the per-batch W
  void* d_alt = nullptr;
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t ev_up[2] = {nullptr, nullptr};
  cudaEvent_t ev_free[2] = {nullptr, nullptr};
  double* h_W = nullptr;
  int h_W_cap = 0;

  // sldg_step as a replayed CUDA graph of one step (two variants: without /
  // with the W history, whose slot comes from a device counter); with merged
  // drifts the graph holds the part of a step between two merged drifts
  // [W history or not + 2 * chained unit (a step between two steps of one call)]
  cudaGraphExec_t step_graph[4] = {nullptr, nullptr, nullptr, nullptr};
  const void* step_graph_buf[4] = {nullptr, nullptr, nullptr, nullptr};  // f and W history they were made for
  const void* step_graph_W[4] = {nullptr, nullptr, nullptr, nullptr};
  long long step_graph_launches[4] = {0, 0, 0, 0};
  bool graphs_off = false;  // a capture failed: steps run eagerly from then on
  int* d_counter = nullptr;

  // state
  double t = 0.0;
  long long step = 0;
  long long launches = 0;
  int x12_shape[2] = {0, 0};  // last fused x pass: CTAs per x-plane, lanes per x1 line pair

  // timing
  bool timing = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<int> ev_kind;  // kind per recorded pair
  size_t ev_used = 0;        // pairs used
  double acc_ms[SLDG_NUM_KINDS] = {0};
  long long acc_n[SLDG_NUM_KINDS] = {0};
};
