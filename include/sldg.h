/*
 * sldg.h -- C ABI of libsldg, a GB300 (sm_103a) implementation of the
 * Strang-split semi-Lagrangian discontinuous Galerkin (SLDG) Vlasov-Poisson
 * step of Einkemmer, arXiv 1803.02143.
 *
 * Problem (Sec. 1, Eq. (vlasov-poisson)):
 *   d_t f + v . grad_x f + E(f) . grad_v f = 0,  div E = int f dv - 1, curl E = 0
 * for f(x1, x2, v1, v2) on a periodic box in x and a bounded box in v.
 *
 * Discretisation (Sec. 2-3): cells of width h_d per direction, f a
 * polynomial of degree l per cell stored by its values at the l+1
 * Gauss-Legendre nodes per direction; each Strang step (Sec. 2)
 *   f^{m+1} = e^{tau/2 A} e^{tau B} e^{tau/2 A} f^m
 * is a sequence of 1D translations projected back onto the cells
 * (Eq. (AB-sldg): out_i = A(theta) in_{i*} + B(theta) in_{i*+1}).
 * Configuration flags select the order-4 composition of Strang steps,
 * merged drifts, or the cubic-spline interpolation of Sec. 3 (the method
 * the paper compares with) in place of the projection.
 *
 * Conventions of every entry point:
 *   - directions d = 0, 1, 2, 3 are x1, x2, v1, v2;
 *   - D_d = ncell[d] * (degree + 1) nodal values per direction, nodal index
 *     i = cell * (degree + 1) + node, node coordinate
 *     lo[d] + (cell + xi_node) * h_d, xi the Gauss-Legendre nodes on [0, 1];
 *   - f is one contiguous device array f[v2][v1][x2][x1] (x1 fastest) of
 *     N = D_0 D_1 D_2 D_3 elements, double (SLDG_FP64) or float (SLDG_FP32);
 *   - x-node arrays (rho, E1, E2) are double [x2][x1], D_0 D_1 elements;
 *   - all device work is issued on the stream given to sldg_init, in
 *     order; entry points that return host data synchronise that stream;
 *   - every function returns SLDG_OK (0) or a negative SLDG_ERR_* code and
 *     never throws or exits; sldg_strerror names the code;
 *   - a context is not thread-safe; distinct contexts are independent.
 *
 * Ownership: f and every buffer passed in are owned by the caller and must
 * stay valid while the context uses them.  The library owns only its
 * context, the projection matrices, rho, E, the spectral tables, reduction
 * partials and (after sldg_record) the checkpoint pool.
 */
#ifndef SLDG_H
#define SLDG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes -------------------------------------------------------- */
#define SLDG_OK 0
#define SLDG_ERR_BAD_CONFIG (-1)  /* invalid or unsupported configuration */
#define SLDG_ERR_BAD_PTR (-2)     /* NULL or misaligned pointer, bad buffer */
#define SLDG_ERR_OOM (-3)         /* device or host allocation failed */
#define SLDG_ERR_CUDA (-4)        /* a CUDA runtime call failed */
#define SLDG_ERR_NONFINITE (-5)   /* a reduction met NaN or Inf in f */
#define SLDG_ERR_UNSUPPORTED (-6) /* size or mode a kernel or entry point does not support */
#define SLDG_ERR_STATE (-7)       /* call out of order (e.g. backward before record) */
#define SLDG_ERR_ARG (-8)         /* invalid scalar argument */

/* ---- enums ----------------------------------------------------------------- */
#define SLDG_FP64 0 /* f stored and swept in double */
#define SLDG_FP32 1 /* f stored and swept in float; matrices built in double and
                       rounded once; rho, Poisson and reductions in double */

/* sldg_config.flags bits */
#define SLDG_FLAG_NATIVE_FP64 1 /* FP64 storage: sweep with FP64 FMA instead of the
                                   default double-float arithmetic on the FP32
                                   pipe (same results to ~1e-15; slower on GB300,
                                   whose FP64 pipe is about 1/64 of FP32) */
#define SLDG_FLAG_NO_XFUSION 2  /* run the X1 and X2 half drifts as two sweeps
                                   instead of one fused pass over each x-plane
                                   (FP32: the same bits; FP64 double-float: the
                                   same arithmetic to its rounding) */
#define SLDG_FLAG_ORDER4 4      /* sldg_step: every step is the fourth-order
                                   triple jump S(w1 tau) S(w0 tau) S(w1 tau) of
                                   Strang steps S, w1 = 1/(2 - 2^(1/3)),
                                   w0 = 1 - 2 w1 < 0 (Sec. 2 cites higher-order
                                   splittings; these are Yoshida's weights);
                                   W_history[m] is W at the first kick of step m */
#define SLDG_FLAG_MERGE_DRIFTS 8 /* sldg_step: consecutive x drifts within one
                                   call (the last drift of a step and the first of
                                   the next, and between ORDER4 sub-steps) run as
                                   one drift of the summed fraction: fewer passes
                                   over f, but not the result of the separate
                                   drifts (the SLDG projection does not compose
                                   exactly), so steps of different calls differ
                                   from one call of all the steps */
#define SLDG_FLAG_SPLINE 16     /* the comparison method of Sec. 3: every sweep is
                                   the cubic-spline advection (periodic cubic
                                   B-spline interpolant of the point values,
                                   evaluated at the shifted points) instead of
                                   the SLDG projection.  Needs degree 0 (one
                                   point per cell: a uniform grid of cell
                                   centres), SLDG_VBC_PERIODIC and 3 <= ncell <= 440
                                   (880 for FP32: two tiles of a line on chip);
                                   rho, Poisson and the diagnostics are those
                                   of the degree-0 grid (midpoint sums).  FP64
                                   storage sweeps in FP64 arithmetic. */
/* sldg_record and sldg_backward differentiate the Strang step of the SLDG
 * sweeps: with ORDER4, MERGE_DRIFTS or SPLINE they return
 * SLDG_ERR_UNSUPPORTED, and so does sldg_sweep_adjoint with SPLINE. */

#define SLDG_VBC_ZERO_INFLOW 0 /* v-sweeps drop source cells outside the box */
#define SLDG_VBC_PERIODIC 1    /* v-sweeps wrap (test mode: exact mass) */

#define SLDG_INIT_LANDAU 0           /* Sec. 4, Eq. (iv-nl); params eps, k1, k2 */
#define SLDG_INIT_TWO_STREAM 1       /* additive two-stream; params eps, k, v0 */
#define SLDG_INIT_TWO_STREAM_PAPER 2 /* Sec. 5, Eq. (iv-tsi); params eps, k, v0 */

/* Kernel classes reported by sldg_timing_read (index into its arrays). */
#define SLDG_K_X1 0
#define SLDG_K_X2 1
#define SLDG_K_V1 2
#define SLDG_K_V2 3
#define SLDG_K_RHO 4
#define SLDG_K_POISSON 5
#define SLDG_K_VMAT 6
#define SLDG_K_OTHER 7
#define SLDG_K_ADJ_X 8
#define SLDG_K_ADJ_V 9
#define SLDG_K_X12 10 /* fused X1, X2 half drifts */
#define SLDG_NUM_KINDS 11

typedef struct {
  int degree;       /* l in 0..3 (dG(l+1)); l+1 nodes per cell and direction */
  int ncell[4];     /* cells per direction, each >= 2 */
  double lo[4];     /* box lower bounds: x1, x2, v1, v2 */
  double hi[4];     /* box upper bounds, hi > lo */
  double dt;        /* time step tau > 0 */
  int precision;    /* SLDG_FP64 or SLDG_FP32 */
  int vbc;          /* SLDG_VBC_ZERO_INFLOW or SLDG_VBC_PERIODIC */
  int poisson_kmax; /* Fourier modes |m_d| <= K_d; < 0 selects
                       K_d = min(ncell_d - 1, (D_d - 1) / 2) */
  int flags;        /* 0 or SLDG_FLAG_* bits */
} sldg_config;

typedef struct {
  double t;        /* simulated time */
  long long step;  /* completed Strang steps */
  double mass;     /* sum w f                       (4D Gauss-Legendre weight w) */
  double l1;       /* sum w |f|                     (Sec. 4, Fig. 4: L1 norm) */
  double l2sq;     /* sum w f^2                     (square of the L2 norm) */
  double kinetic;  /* 1/2 sum w (v1^2 + v2^2) f */
  double electric; /* W = 1/2 sum_x w_x (E1^2 + E2^2), E of the current f */
  double total;    /* kinetic + electric            (Sec. 4: energy) */
} sldg_diag;

typedef struct sldg_ctx sldg_ctx;

/* Name of a status code (static string, never NULL). */
const char* sldg_strerror(int code);

/* ABI version of this header (increments on any signature change). */
int sldg_abi_version(void);

/* ---- life cycle -------------------------------------------------------------
 * sldg_init: validate cfg, bind the caller's device array f_dev (N elements of
 * the configured precision, 16-byte aligned) and the CUDA stream (a
 * cudaStream_t; NULL is the legacy default stream), build the Gauss-Legendre
 * nodes, the x-sweep matrices (one pair per v-node, Sec. 3: "precomputed") and
 * the spectral tables.  f_dev is not read or written here.
 * Errors: BAD_CONFIG (degree outside 0..3, ncell < 2, hi <= lo, dt <= 0,
 * unknown precision/vbc, unknown flag bits, SLDG_FLAG_SPLINE without degree
 * 0, periodic v and ncell >= 3, a line too long for on-chip staging),
 * BAD_PTR (cfg or out NULL, f_dev NULL or misaligned), OOM, CUDA. */
int sldg_init(const sldg_config* cfg, void* f_dev, void* stream, sldg_ctx** out);

/* Release everything the library owns; f_dev is untouched.  NULL is a no-op. */
void sldg_destroy(sldg_ctx* ctx);

/* Number of nodal values N of the context's grid (0 for NULL). */
long long sldg_numel(const sldg_ctx* ctx);

/* Rebind the context to another caller-owned array of the same size and
 * precision (e.g. a resumed state).  BAD_PTR if NULL or misaligned. */
int sldg_bind(sldg_ctx* ctx, void* f_dev);

/* ---- state --------------------------------------------------------------------
 * sldg_set_initial: evaluate an initial value at the nodes into f (nodal
 * interpolation, Sec. 2: values at the Gauss-Legendre points), reset t and
 * the step counter.  kind SLDG_INIT_*; params[0..2] as listed there.
 * Errors: ARG (unknown kind, nparams < 3), BAD_PTR (params NULL). */
int sldg_set_initial(sldg_ctx* ctx, int kind, const double* params, int nparams);

/* Copy f to/from a caller buffer of N elements of the context's precision:
 * on_device != 0 for device memory, 0 for host memory (pinned host memory
 * gives asynchronous copies).  sldg_get_f synchronises the stream when dst is
 * host memory.  sldg_set_f also sets t and the step counter. */
int sldg_get_f(sldg_ctx* ctx, void* dst, int on_device);
int sldg_set_f(sldg_ctx* ctx, const void* src, int on_device, double t, long long step);

/* ---- the hot path ------------------------------------------------------------
 * sldg_step: advance f in place by nsteps Strang steps (Sec. 2):
 *   X1(tau/2) X2(tau/2) | rho = Q f, E = L rho | V1(tau E1) V2(tau E2) | X1(tau/2) X2(tau/2)
 * with E frozen over the kick (Sec. 2: the acceleration leaves rho
 * invariant); with SLDG_FLAG_ORDER4 / SLDG_FLAG_MERGE_DRIFTS the
 * compositions those flags describe.  If W_history (host, nsteps doubles)
 * is non-NULL it receives the electric energy W(E) of each step's (first)
 * kick field and the call synchronises the stream; otherwise the call is
 * asynchronous.  FP64 storage with double-float sweeps: f holds IEEE doubles
 * before and after the call; between the steps of one call the state stays
 * in the sweeps' double-float pairs, so one call of n steps and n calls of
 * one step agree to rounding (about 2^-47 relative per step), not bit for bit.
 * Errors: ARG (nsteps < 0), CUDA. */
int sldg_step(sldg_ctx* ctx, int nsteps, double* W_history);

/* One Strang step for each of nbatch states that live in host memory: batch
 * b is the N elements (context precision) at host_f + b * batch_stride_bytes
 * (stride 0: the same host state every time); W of its step goes to
 * W_out[b] (host, nbatch doubles).  Batch b+1 is copied host-to-device on a
 * second stream, into a library-owned second state buffer, while batch b
 * is stepped on the context's stream, so the copies and the steps overlap;
 * host_f should be pinned (page-locked) memory for the copies to run at
 * full speed and asynchronously.  On return f holds the stepped state of
 * the last batch and t, step have advanced by one step.  Synchronises.
 * Errors: BAD_PTR, ARG (nbatch < 1 or a negative stride), OOM, CUDA. */
int sldg_step_host_batches(sldg_ctx* ctx, const void* host_f, long long batch_stride_bytes,
                           int nbatch, double* W_out);

/* One 1D sweep in place along direction dim (Sec. 3, Eq. (1d-advection): the
 * one function "executed multiple times with different parameters"):
 *   dim 0, 1: shift a = v_{dim}(node) * dt * frac, periodic in x;
 *   dim 2, 3: shift a = E_{dim-2}(x-node) * dt * frac with the context's
 *             current field (sldg_compute_fields or sldg_set_field).
 * The matrices for frac are rebuilt on the device when frac changes.
 * Errors: ARG (dim outside 0..3), STATE (v-sweep before any field). */
int sldg_sweep(sldg_ctx* ctx, int dim, double frac);

/* The free-streaming half of a Strang step on its own (Sec. 2, e^{tau A} =
 * e^{tau A2} e^{tau A1}): X1 then X2 in place on f, each line shifted by its
 * velocity node times dt * frac, periodic in x.  These are the kernels and
 * the launch configuration of the drifts inside sldg_step (one fused pass
 * over each x-plane where the layout allows it, else the two sweeps), with
 * IEEE values in and out.  Errors: ARG (frac not finite), CUDA. */
int sldg_drift(sldg_ctx* ctx, double frac);

/* rho = Q f (v-quadrature, Sec. 2: rho = int g dv) and E = L rho (spectral
 * Poisson, Sec. 3 "FFTW"; dense map on the nodes with the mean mode removed)
 * of the current f; stores them in the context. */
int sldg_compute_fields(sldg_ctx* ctx);

/* Overwrite the context's field with E1, E2 (D_0 D_1 doubles each; device
 * memory if on_device, else host).  Used for free streaming (E = 0) and for
 * testing the v-sweeps against a prescribed field. */
int sldg_set_field(sldg_ctx* ctx, const double* E1, const double* E2, int on_device);

/* Copy the context's rho, E1, E2 (each D_0 D_1 doubles; any pointer may be
 * NULL) to device (on_device != 0) or host memory (synchronises). */
int sldg_fields(sldg_ctx* ctx, double* rho, double* E1, double* E2, int on_device);

/* Diagnostics of the current f (Sec. 4, Fig. 4; Sec. 5, Fig. 5) with
 * compensated FP64 reductions; recomputes the field of the current f.
 * Synchronises.  Returns NONFINITE (and fills out) if f holds NaN or Inf. */
int sldg_diagnostics(sldg_ctx* ctx, sldg_diag* out);

/* ---- adjoint -----------------------------------------------------------------
 * Transposed sweep in place on lam (N elements, context precision, device):
 * lam <- S(dim)^T lam, the transpose of the projected translation (the
 * adjoint of Eq. (AB-sldg): in_bar_{i*} += A^T out_bar_i,
 * in_bar_{i*+1} += B^T out_bar_i).  For dim 2, 3, if g (the forward input of
 * that sweep, N elements) and Ebar (device, D_0 D_1 doubles) are non-NULL,
 * adds to Ebar the derivative of <lam_out, S(E) g> with respect to E at every
 * x-node (dA/dtheta, dB/dtheta times dt*frac/h_v, summed over v).
 * Errors: ARG, BAD_PTR, STATE. */
int sldg_sweep_adjoint(sldg_ctx* ctx, int dim, double frac, void* lam, const void* g,
                       double* Ebar);

/* Run nsteps Strang steps from the current f like sldg_step while keeping a
 * checkpoint of f every ckpt_every steps in a library-owned device pool
 * (ceil(nsteps / ckpt_every) copies of f), and record W of each step
 * (W_history, host, nullable).  Prepares sldg_backward.  The pool, the W
 * history and sldg_backward's working copies stay allocated until
 * sldg_destroy or a recording that needs a larger pool (which releases the
 * backward's copies first if the pool does not fit beside them).
 * Errors: ARG, OOM (the pool does not fit), UNSUPPORTED (SLDG_FLAG_ORDER4,
 * SLDG_FLAG_MERGE_DRIFTS or SLDG_FLAG_SPLINE), CUDA. */
int sldg_record(sldg_ctx* ctx, int nsteps, int ckpt_every, double* W_history);

/* J = sum_m c_m W(E^m) of the last sldg_record, c_m = cW[m] (host, ncW =
 * nsteps doubles) or dt if cW is NULL: the time-integrated electric energy
 * for c_m = dt (a compensated sum of the recorded W history), to *J_out.
 * Synchronises.  Errors: BAD_PTR, STATE (no record), ARG (ncW differs from
 * the recorded step count), CUDA. */
int sldg_objective(sldg_ctx* ctx, const double* cW, int ncW, double* J_out);

/* Reverse pass of the last sldg_record: gradient of
 *   J = sum_m c_m W(E^m),   c_m = cW[m] (host, ncW = nsteps doubles) or dt if NULL,
 * (the time-integrated electric energy for c_m = dt) with respect to every
 * nodal value of the recorded initial f, written to grad (device, N elements
 * of the context precision).  J_out (host, nullable) receives J.  f is left
 * at the recorded final state.
 * Memory: besides the checkpoint pool, two copies of f for the forward
 * intermediates of one step and up to 2 ckpt_every + 1 recomputation slots
 * (copies of f), as many as fit in the free device memory less a margin
 * (and at most the limit of sldg_set_slot_limit).  With 2 S + 1 slots for a
 * segment of S steps, one forward pass keeps every step's intermediates
 * (the inputs of V1 and V2 and the kick field); with S - 1, the segment's
 * states are kept and each step's intermediates rebuilt; with fewer, the
 * segment is bisected recursively and its states are recomputed about
 * log2(ckpt_every) times; with one slot, from the checkpoint for every
 * step.  The gradient is the same whatever the number of slots (the same
 * arithmetic, only repeated).  On FP64 storage with double-float sweeps the
 * adjoint is carried in grad as double-float pairs; the last kernel the call
 * queues converts it to IEEE doubles.
 * Errors: STATE (no record), BAD_PTR, ARG (ncW differs from the recorded
 * step count), OOM (not even one slot fits), UNSUPPORTED (SLDG_FLAG_ORDER4,
 * SLDG_FLAG_MERGE_DRIFTS or SLDG_FLAG_SPLINE), CUDA. */
int sldg_backward(sldg_ctx* ctx, const double* cW, int ncW, void* grad, double* J_out);

/* Upper bound on the recomputation slots of sldg_backward (0 = as many as a
 * segment can use and the device has room for).  Errors: BAD_PTR, ARG. */
int sldg_set_slot_limit(sldg_ctx* ctx, int max_slots);

/* Strang steps recomputed by the last sldg_backward and the slots it held
 * (either pointer nullable).  Errors: BAD_PTR. */
int sldg_backward_stats(const sldg_ctx* ctx, long long* recomputed_steps, int* slots);

/* sum_n grad[n] * d f0[n] / d params[0] for an initial value of kind
 * SLDG_INIT_* (the derivative with respect to the perturbation amplitude),
 * with grad a device array of N elements in the context precision; result to
 * *out (host).  Synchronises. */
int sldg_initial_param_grad(sldg_ctx* ctx, int kind, const double* params, int nparams,
                            const void* grad, double* out);

/* ---- allocation-free charge density --------------------------------------------
 * The paper has no counterpart of this entry point; it serves callers that
 * cannot allocate device memory.  cudaMalloc and cudaFree synchronise the
 * whole device and take memory outside the caller's own accounting, so code
 * running in a latency-bound per-step loop, code whose device memory is
 * owned by another allocator (a framework's caching pool) and code under a
 * fixed memory budget cannot call them, and sldg_init allocates.
 *
 * rho(x) = sum_v w_v f[v][x] of the grid described by cfg (degree, ncell,
 * lo, hi and precision are read; nothing is kept), f_dev the caller's device
 * array in the layout of sldg_init, rho_dev the caller's device array of
 * D_0 D_1 doubles, work issued on `stream` (a cudaStream_t; NULL is the
 * legacy default stream).  Same values as sldg_compute_fields' rho to
 * rounding.  No device memory is allocated: the partial sums live in a fixed
 * 4 MiB array inside the library, held by every device that loads it until
 * exit.  The first call on each device (with that device current) looks up
 * that array's device address; make that call before any stream capture.
 * Nothing has to start at zero: each call writes every partial sum before
 * it reads it and overwrites all of rho_dev.  Every call reuses the same
 * array, so calls that overlap on the GPU (other streams, other host
 * threads) race and must be ordered by the caller.
 * A CUDA error left pending by the caller's earlier work is cleared on
 * entry (it would otherwise read as this call's launch failure).
 * Errors: BAD_PTR, BAD_CONFIG (every configuration sldg_init rejects),
 * UNSUPPORTED (x-plane D_0 D_1 above 2^19 nodes, or a v-chunk beyond shared
 * memory), CUDA. */
int sldg_rho_noalloc(const sldg_config* cfg, const void* f_dev, double* rho_dev, void* stream);

/* ---- measurement ---------------------------------------------------------------
 * Kernel launches issued by this context since init (all entry points). */
long long sldg_launch_count(const sldg_ctx* ctx);

/* Launch shape of the last fused X1 X2 pass this context ran (either pointer
 * nullable): the CTAs that share one x-plane (a thread-block cluster) and
 * the lanes given to each pair of x1 lines in its X1 phase (32: whole warps;
 * fewer: several line pairs per warp).  Both 0 before the first fused pass.
 * Errors: BAD_PTR. */
int sldg_x_pass_shape(const sldg_ctx* ctx, int* cluster_ctas, int* lanes_per_line_pair);

/* enable != 0: bracket every subsequent kernel launch with CUDA events on the
 * context's stream, accumulated per kernel class SLDG_K_*; 0 stops; both
 * clear the accumulators. */
int sldg_timing(sldg_ctx* ctx, int enable);

/* Synchronise and report per class: total milliseconds (ms[SLDG_NUM_KINDS])
 * and launches (count[SLDG_NUM_KINDS]); either pointer may be NULL. */
int sldg_timing_read(sldg_ctx* ctx, double* ms, long long* count);

#ifdef __cplusplus
}
#endif
#endif /* SLDG_H */
