/*
 * sldg_oracle.c -- plain, slow FP64 CPU oracle for the semi-Lagrangian
 * discontinuous Galerkin (SLDG) Vlasov-Poisson step of Einkemmer,
 * "A comparison of semi-Lagrangian discontinuous Galerkin and spline based
 * Vlasov solvers in four dimensions" (arXiv 1803.02143).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent checker for the
 * CUDA library: only the tests, the smoke check and the benchmark's CPU
 * baseline leg load it.  It shares no code, header, table or constant
 * generator with the CUDA path; the product never links or calls it.
 *
 * Everything is FP64, plain loops, in the order the paper states the method.
 * OpenMP (when compiled with it) only distributes independent lines or
 * independent output nodes; every sum runs serially in a fixed order, so the
 * results do not depend on the thread count.
 *
 * Conventions (shared with the CUDA library by specification only):
 *   - directions d = 0,1,2,3 are x1, x2, v1, v2;
 *   - direction d has nc[d] cells of width h_d = (hi[d]-lo[d])/nc[d] and
 *     D_d = nc[d]*(deg+1) nodal values, index i = cell*(deg+1) + node;
 *   - node coordinate z = lo + (cell + xi_j) h with xi_j the Gauss-Legendre
 *     nodes on [0,1] (Sec. 3, the nodal degrees of freedom);
 *   - f is stored f[v2][v1][x2][x1], x1 fastest;
 *   - x is periodic; v is zero-inflow (vbc = 0) or periodic (vbc = 1).
 *
 * Readings of the paper this oracle fixes (the paper is silent on them):
 *   - each x-sweep shifts every line by the velocity of its own v-node, each
 *     v-sweep by tau*E at its own x-node (the 1D advection "executed multiple
 *     times with different parameters", Sec. 3);
 *   - the Poisson map is a dense spectral map on the Gauss-Legendre nodes,
 *     mean mode removed, |m_d| <= K_d (see orc_poisson);
 *   - the electric energy is W = 1/2 sum_x w_x (E1^2 + E2^2).
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAXN 8 /* at most 8 nodes per cell (degree <= 7) */

typedef struct {
  int deg;        /* polynomial degree l per cell; l+1 Gauss-Legendre nodes */
  int nc[4];      /* cells per direction x1, x2, v1, v2 */
  double lo[4];   /* lower domain bound per direction */
  double hi[4];   /* upper domain bound per direction */
  double dt;      /* time step tau */
  int vbc;        /* 0: zero inflow in v, 1: periodic in v */
  int kmax;       /* Poisson modes per direction, < 0: min(nc-1, (D-1)/2) */
  int spline;     /* 1: sweeps by cubic-spline interpolation (degree 0 grid,
                     periodic in every direction), see orc_spline_line */
} orc_grid;

/* ------------------------------------------------------------------------ */
/* Gauss-Legendre nodes and weights on [0,1] (Sec. 3: nodal dofs at the      */
/* Gauss-Legendre points).  Newton's method on the Legendre polynomial P_n    */
/* evaluated by its three-term recurrence.  Weights sum to one.              */
/* ------------------------------------------------------------------------ */
static void legendre_pn(int n, double x, double* pn, double* pnm1) {
  double p0 = 1.0, p1 = x;
  if (n == 0) { *pn = 1.0; *pnm1 = 0.0; return; }
  for (int k = 1; k < n; ++k) {
    double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
    p0 = p1;
    p1 = p2;
  }
  *pn = p1;
  *pnm1 = p0;
}

int orc_gauss_legendre(int n, double* xi, double* w) {
  if (n < 1 || n > ORC_MAXN) return -1;
  for (int i = 0; i < n; ++i) {
    double x = cos(M_PI * (i + 0.75) / (n + 0.5)); /* i-th root, descending */
    double pn, pnm1, dp;
    for (int it = 0; it < 100; ++it) {
      legendre_pn(n, x, &pn, &pnm1);
      dp = n * (x * pn - pnm1) / (x * x - 1.0);
      double dx = pn / dp;
      x -= dx;
      if (fabs(dx) < 1e-16) break;
    }
    legendre_pn(n, x, &pn, &pnm1);
    dp = n * (x * pn - pnm1) / (x * x - 1.0);
    xi[i] = 0.5 * (1.0 - x);                   /* ascending on [0,1] */
    w[i] = 1.0 / ((1.0 - x * x) * dp * dp);    /* (2/((1-x^2)P'^2)) / 2 */
  }
  return 0;
}

/* Lagrange basis on the nodes xi: phi_j(xi_l) = delta_jl. */
static double lag(int n, const double* xi, int j, double t) {
  double p = 1.0;
  for (int m = 0; m < n; ++m)
    if (m != j) p *= (t - xi[m]) / (xi[j] - xi[m]);
  return p;
}

static double lagd(int n, const double* xi, int j, double t) {
  double s = 0.0;
  for (int k = 0; k < n; ++k) {
    if (k == j) continue;
    double p = 1.0 / (xi[j] - xi[k]);
    for (int m = 0; m < n; ++m)
      if (m != j && m != k) p *= (t - xi[m]) / (xi[j] - xi[m]);
    s += p;
  }
  return s;
}

double orc_lagrange(int n, const double* xi, int j, double t) { return lag(n, xi, j, t); }
double orc_lagrange_d(int n, const double* xi, int j, double t) { return lagd(n, xi, j, t); }

/* ------------------------------------------------------------------------ */
/* Projection matrices of Eq. (AB-sldg).                                     */
/*                                                                           */
/* A translation by a = (s + theta) h, s integer, theta in [0,1), moves the  */
/* part t < theta of target cell c (local coordinate t in [0,1]) onto cell    */
/* c-s-1 at local coordinate t+1-theta, and the part t >= theta onto cell     */
/* c-s at t-theta.  The L2 projection onto degree-l polynomials with the     */
/* Lagrange basis at the Gauss-Legendre nodes has the diagonal mass matrix    */
/* h w_j (Sec. 2, the projection P; Sec. 3, Eq. (AB-sldg)), hence           */
/*   A_jl = (1/w_j) int_0^theta  phi_j(t) phi_l(t+1-theta) dt   (cell c-s-1) */
/*   B_jl = (1/w_j) int_theta^1  phi_j(t) phi_l(t-theta)   dt   (cell c-s)   */
/* Each integrand has degree 2l, so (l+1)-point Gauss-Legendre on the       */
/* sub-interval is exact (Sec. 2: quadrature computes the projection         */
/* "analytically").  The derivatives with respect to theta follow from the   */
/* Leibniz rule:                                                             */
/*   A'_jl = (1/w_j)[ phi_j(theta) phi_l(1) - int_0^theta phi_j phi_l'(t+1-theta) ] */
/*   B'_jl = (1/w_j)[-phi_j(theta) phi_l(0) - int_theta^1 phi_j phi_l'(t-theta)  ] */
/* Matrices are row-major, A[j*(l+1) + l'].                                  */
/* ------------------------------------------------------------------------ */
int orc_matrices(int deg, double theta, double* A, double* B, double* dA, double* dB) {
  int n = deg + 1;
  double xi[ORC_MAXN], w[ORC_MAXN];
  if (orc_gauss_legendre(n, xi, w) != 0) return -1;
  for (int j = 0; j < n; ++j) {
    for (int l = 0; l < n; ++l) {
      double a = 0.0, b = 0.0, da = 0.0, db = 0.0;
      for (int q = 0; q < n; ++q) {
        double ta = theta * xi[q];                  /* node of [0, theta] */
        double tb = theta + (1.0 - theta) * xi[q];  /* node of [theta, 1] */
        a += theta * w[q] * lag(n, xi, j, ta) * lag(n, xi, l, ta + 1.0 - theta);
        b += (1.0 - theta) * w[q] * lag(n, xi, j, tb) * lag(n, xi, l, tb - theta);
        da += theta * w[q] * lag(n, xi, j, ta) * lagd(n, xi, l, ta + 1.0 - theta);
        db += (1.0 - theta) * w[q] * lag(n, xi, j, tb) * lagd(n, xi, l, tb - theta);
      }
      A[j * n + l] = a / w[j];
      B[j * n + l] = b / w[j];
      if (dA) dA[j * n + l] = (lag(n, xi, j, theta) * lag(n, xi, l, 1.0) - da) / w[j];
      if (dB) dB[j * n + l] = (-lag(n, xi, j, theta) * lag(n, xi, l, 0.0) - db) / w[j];
    }
  }
  return 0;
}

/* Split a shift a (in units of h) into s = floor(a/h) and theta in [0,1). */
static void split_shift(double a, double h, long* s, double* theta) {
  double sigma = a / h;
  double sf = floor(sigma);
  *s = (long)sf;
  *theta = sigma - sf;
  if (*theta >= 1.0) { /* sigma just below an integer rounded up */
    *theta = 0.0;
    *s += 1;
  }
}

static long wrap(long k, long nc) {
  long r = k % nc;
  return r < 0 ? r + nc : r;
}

/* ------------------------------------------------------------------------ */
/* The one-dimensional advection u^{m+1}(x) = u^m(x - a) of Eq. (1d-         */
/* advection), projected: for every target cell c                           */
/*   out[c] = A(theta) in[c-s-1] + B(theta) in[c-s]      (Eq. (AB-sldg))     */
/* with source cells wrapped (periodic) or dropped (zero inflow).            */
/* ------------------------------------------------------------------------ */
void orc_advect_line(int deg, int nc, double h, double a, int periodic,
                     const double* in, double* out) {
  int n = deg + 1;
  long s;
  double theta, A[ORC_MAXN * ORC_MAXN], B[ORC_MAXN * ORC_MAXN];
  split_shift(a, h, &s, &theta);
  orc_matrices(deg, theta, A, B, NULL, NULL);
  for (long c = 0; c < nc; ++c) {
    long ka = c - s - 1, kb = c - s;
    const double* ua = NULL;
    const double* ub = NULL;
    if (periodic) {
      ua = in + wrap(ka, nc) * n;
      ub = in + wrap(kb, nc) * n;
    } else {
      if (ka >= 0 && ka < nc) ua = in + ka * n;
      if (kb >= 0 && kb < nc) ub = in + kb * n;
    }
    for (int j = 0; j < n; ++j) {
      double acc = 0.0;
      for (int l = 0; l < n; ++l) {
        if (ua) acc += A[j * n + l] * ua[l];
        if (ub) acc += B[j * n + l] * ub[l];
      }
      out[c * n + j] = acc;
    }
  }
}

/* Transpose of orc_advect_line: lam_in = S(a)^T lam_out. */
void orc_advect_line_adj(int deg, int nc, double h, double a, int periodic,
                         const double* lam_out, double* lam_in) {
  int n = deg + 1;
  long s;
  double theta, A[ORC_MAXN * ORC_MAXN], B[ORC_MAXN * ORC_MAXN];
  split_shift(a, h, &s, &theta);
  orc_matrices(deg, theta, A, B, NULL, NULL);
  for (long i = 0; i < (long)nc * n; ++i) lam_in[i] = 0.0;
  for (long c = 0; c < nc; ++c) {
    long ka = c - s - 1, kb = c - s;
    double* ua = NULL;
    double* ub = NULL;
    if (periodic) {
      ua = lam_in + wrap(ka, nc) * n;
      ub = lam_in + wrap(kb, nc) * n;
    } else {
      if (ka >= 0 && ka < nc) ua = lam_in + ka * n;
      if (kb >= 0 && kb < nc) ub = lam_in + kb * n;
    }
    for (int j = 0; j < n; ++j) {
      for (int l = 0; l < n; ++l) {
        if (ua) ua[l] += A[j * n + l] * lam_out[c * n + j];
        if (ub) ub[l] += B[j * n + l] * lam_out[c * n + j];
      }
    }
  }
}

/* d/da <lam_out, S(a) in> for fixed s (theta = a/h - s, dtheta/da = 1/h). */
double orc_advect_line_dshift(int deg, int nc, double h, double a, int periodic,
                              const double* lam_out, const double* in) {
  int n = deg + 1;
  long s;
  double theta, A[ORC_MAXN * ORC_MAXN], B[ORC_MAXN * ORC_MAXN];
  double dA[ORC_MAXN * ORC_MAXN], dB[ORC_MAXN * ORC_MAXN];
  split_shift(a, h, &s, &theta);
  orc_matrices(deg, theta, A, B, dA, dB);
  double acc = 0.0;
  for (long c = 0; c < nc; ++c) {
    long ka = c - s - 1, kb = c - s;
    const double* ua = NULL;
    const double* ub = NULL;
    if (periodic) {
      ua = in + wrap(ka, nc) * n;
      ub = in + wrap(kb, nc) * n;
    } else {
      if (ka >= 0 && ka < nc) ua = in + ka * n;
      if (kb >= 0 && kb < nc) ub = in + kb * n;
    }
    for (int j = 0; j < n; ++j) {
      double d = 0.0;
      for (int l = 0; l < n; ++l) {
        if (ua) d += dA[j * n + l] * ua[l];
        if (ub) d += dB[j * n + l] * ub[l];
      }
      acc += lam_out[c * n + j] * d;
    }
  }
  return acc / h;
}

/* ------------------------------------------------------------------------ */
/* Grid helpers.                                                             */
/* ------------------------------------------------------------------------ */
static long dimlen(const orc_grid* g, int d) { return (long)g->nc[d] * (g->deg + 1); }
static double cellw(const orc_grid* g, int d) { return (g->hi[d] - g->lo[d]) / g->nc[d]; }

static void strides(const orc_grid* g, long D[4], long S[4]) {
  for (int d = 0; d < 4; ++d) D[d] = dimlen(g, d);
  S[0] = 1;
  S[1] = D[0];
  S[2] = D[0] * D[1];
  S[3] = D[0] * D[1] * D[2];
}

static double node_coord(const orc_grid* g, int d, long i, const double* xi) {
  int n = g->deg + 1;
  return g->lo[d] + ((double)(i / n) + xi[i % n]) * cellw(g, d);
}

static double node_weight(const orc_grid* g, int d, long i, const double* w) {
  return cellw(g, d) * w[i % (g->deg + 1)];
}

long orc_numel(const orc_grid* g) {
  return dimlen(g, 0) * dimlen(g, 1) * dimlen(g, 2) * dimlen(g, 3);
}

/* ------------------------------------------------------------------------ */
/* The spline method of Sec. 3 for the same 1D advection, on n equidistant   */
/* points x_i (spacing h, periodic): the interpolant                          */
/*   u~(x) = sum_k w_k S(x - x_k),                                            */
/*   6 S(x) = 4 - 6 (x/h)^2 + 3 |x/h|^3 (|x| <= h), (2 - |x/h|)^3 (h <= |x|    */
/*   <= 2h), 0 beyond,                                                        */
/* has coefficients from the cyclic tridiagonal system                        */
/*   (w_{i-1} + 4 w_i + w_{i+1}) / 6 = u_i   (indices mod n),                 */
/* and the new values are u~(x_i - a).  The cyclic system is solved with the  */
/* Thomas algorithm on the tridiagonal part and a rank-one (Sherman-          */
/* Morrison) correction for the two corner entries.                           */
/* ------------------------------------------------------------------------ */
static void thomas(long n, const double* sub, const double* dia, const double* sup,
                   const double* rhs, double* x, double* cp) {
  /* forward elimination (cp: modified super-diagonal), back substitution */
  double den = dia[0];
  cp[0] = sup[0] / den;
  x[0] = rhs[0] / den;
  for (long i = 1; i < n; ++i) {
    den = dia[i] - sub[i] * cp[i - 1];
    cp[i] = sup[i] / den;
    x[i] = (rhs[i] - sub[i] * x[i - 1]) / den;
  }
  for (long i = n - 2; i >= 0; --i) x[i] -= cp[i] * x[i + 1];
}

int orc_spline_coeffs(long n, const double* u, double* w) {
  if (n < 3) return -1;
  double* sub = (double*)malloc((size_t)n * 6 * sizeof(double));
  if (!sub) return -3;
  double *dia = sub + n, *sup = dia + n, *y = sup + n, *z = y + n, *cp = z + n;
  /* A = B + p q^T with p = (g, 0, .., 0, 1/6), q = (1, 0, .., 0, (1/6)/g),
     g = -4/6: B is tridiagonal with its two corner diagonal entries changed */
  const double off = 1.0 / 6.0, d = 4.0 / 6.0, g = -d;
  for (long i = 0; i < n; ++i) {
    sub[i] = off;
    dia[i] = d;
    sup[i] = off;
  }
  dia[0] = d - g;
  dia[n - 1] = d - off * off / g;
  thomas(n, sub, dia, sup, u, y, cp);
  for (long i = 0; i < n; ++i) w[i] = 0.0;
  w[0] = g;
  w[n - 1] = off;
  thomas(n, sub, dia, sup, w, z, cp);
  const double qy = y[0] + off / g * y[n - 1], qz = z[0] + off / g * z[n - 1];
  const double fac = qy / (1.0 + qz);
  for (long i = 0; i < n; ++i) w[i] = y[i] - fac * z[i];
  free(sub);
  return 0;
}

/* out_i = u~(x_i - a): with a/h = s + theta (s integer, 0 <= theta < 1) the
   point x_i - a lies theta h before x_{i-s}, and the four B-splines there
   give  6 out_i = theta^3 w_{i-s-2} + (4 - 6 (1-theta)^2 + 3 (1-theta)^3)
   w_{i-s-1} + (4 - 6 theta^2 + 3 theta^3) w_{i-s} + (1-theta)^3 w_{i-s+1}. */
int orc_spline_line(long n, double h, double a, const double* u, double* out) {
  double* w = (double*)malloc((size_t)n * sizeof(double));
  if (!w) return -3;
  int rc = orc_spline_coeffs(n, u, w);
  if (rc) {
    free(w);
    return rc;
  }
  long s;
  double th;
  split_shift(a, h, &s, &th);
  const double om = 1.0 - th;
  const double b0 = th * th * th, b1 = 4.0 - 6.0 * om * om + 3.0 * om * om * om;
  const double b2 = 4.0 - 6.0 * th * th + 3.0 * th * th * th, b3 = om * om * om;
  for (long i = 0; i < n; ++i)
    out[i] = (b0 * w[wrap(i - s - 2, n)] + b1 * w[wrap(i - s - 1, n)] + b2 * w[wrap(i - s, n)] +
              b3 * w[wrap(i - s + 1, n)]) / 6.0;
  free(w);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* A sweep: the 1D advection applied to every line along direction d.        */
/*   d = 0 (x1): shift a = v1(node) * dt * frac, periodic  (e^{tau A_1})     */
/*   d = 1 (x2): shift a = v2(node) * dt * frac, periodic  (e^{tau A_2})     */
/*   d = 2 (v1): shift a = E1(x)    * dt * frac            (e^{tau B}, v1)   */
/*   d = 3 (v2): shift a = E2(x)    * dt * frac            (e^{tau B}, v2)   */
/* (Sec. 2: e^{tau A} g = g(x - tau v, v), e^{tau B} g = g(x, v - tau E),    */
/*  each split into commuting 1D advections.)                                */
/* mode 0: forward out = S in;  mode 1: adjoint out = S^T in, and when Ebar  */
/* is given, Ebar[x] += (dt*frac) d/da <in, S(a) g>  summed over its lines.  */
/* ------------------------------------------------------------------------ */
static int sweep_impl(const orc_grid* g, int d, const double* Ed, double frac,
                      const double* fin, double* fout, int mode, const double* gfwd,
                      double* Ebar) {
  int n = g->deg + 1;
  double xi[ORC_MAXN], w[ORC_MAXN];
  long D[4], S[4];
  if (d < 0 || d > 3 || n > ORC_MAXN) return -1;
  if (d >= 2 && !Ed) return -1;
  orc_gauss_legendre(n, xi, w);
  strides(g, D, S);
  long N = D[0] * D[1] * D[2] * D[3];
  long len = D[d], nlines = N / len;
  int o[3], k = 0;
  for (int e = 0; e < 4; ++e)
    if (e != d) o[k++] = e;
  int periodic = (d < 2) ? 1 : (g->vbc == 1);
  double h = cellw(g, d);
  if (g->spline && (mode != 0 || !periodic || g->deg != 0)) return -1;
  long Dx = D[0] * D[1];
  /* Ebar contributions are kept per line so the per-x-node sum can run in a
     fixed order afterwards, independent of the thread count. */
  double* lined = (Ebar && mode == 1) ? (double*)calloc((size_t)nlines, sizeof(double)) : NULL;
  int failed = 0;

#pragma omp parallel
  {
    double* a_in = (double*)malloc((size_t)len * sizeof(double));
    double* a_out = (double*)malloc((size_t)len * sizeof(double));
    double* a_g = gfwd ? (double*)malloc((size_t)len * sizeof(double)) : NULL;
#pragma omp for schedule(static)
    for (long L = 0; L < nlines; ++L) {
      long idx[4];
      long r = L;
      idx[o[0]] = r % D[o[0]]; r /= D[o[0]];
      idx[o[1]] = r % D[o[1]]; r /= D[o[1]];
      idx[o[2]] = r;
      idx[d] = 0;
      long base = idx[0] * S[0] + idx[1] * S[1] + idx[2] * S[2] + idx[3] * S[3];
      double a;
      if (d == 0) a = node_coord(g, 2, idx[2], xi) * g->dt * frac;
      else if (d == 1) a = node_coord(g, 3, idx[3], xi) * g->dt * frac;
      else a = Ed[idx[1] * D[0] + idx[0]] * g->dt * frac;
      for (long i = 0; i < len; ++i) a_in[i] = fin[base + i * S[d]];
      if (mode == 0 && g->spline) {
        if (orc_spline_line(len, h, a, a_in, a_out) != 0) {
#pragma omp atomic write
          failed = 1;
        }
      } else if (mode == 0) {
        orc_advect_line(g->deg, g->nc[d], h, a, periodic, a_in, a_out);
      } else {
        orc_advect_line_adj(g->deg, g->nc[d], h, a, periodic, a_in, a_out);
        if (lined) {
          for (long i = 0; i < len; ++i) a_g[i] = gfwd[base + i * S[d]];
          lined[L] = g->dt * frac *
                     orc_advect_line_dshift(g->deg, g->nc[d], h, a, periodic, a_in, a_g);
        }
      }
      for (long i = 0; i < len; ++i) fout[base + i * S[d]] = a_out[i];
    }
    free(a_in);
    free(a_out);
    free(a_g);
  }
  if (lined) {
    /* line L of a v-sweep covers x-node (idx[0], idx[1]) = (L % D0, (L/D0) % D1) */
    for (long L = 0; L < nlines; ++L) Ebar[L % Dx] += lined[L];
    free(lined);
  }
  return failed ? -1 : 0;
}

int orc_sweep(const orc_grid* g, int d, const double* Ed, double frac, const double* fin,
              double* fout) {
  return sweep_impl(g, d, Ed, frac, fin, fout, 0, NULL, NULL);
}

int orc_sweep_adj(const orc_grid* g, int d, const double* Ed, double frac,
                  const double* lam_out, double* lam_in, const double* gfwd, double* Ebar) {
  return sweep_impl(g, d, Ed, frac, lam_out, lam_in, 1, gfwd, Ebar);
}

/* ------------------------------------------------------------------------ */
/* Compensated (Neumaier) summation, used for every reduction below.         */
/* ------------------------------------------------------------------------ */
typedef struct { double s, c; } ksum;
static void kadd(ksum* k, double x) {
  double t = k->s + x;
  if (fabs(k->s) >= fabs(x)) k->c += (k->s - t) + x;
  else k->c += (x - t) + k->s;
  k->s = t;
}
static double kval(const ksum* k) { return k->s + k->c; }

/* ------------------------------------------------------------------------ */
/* Charge density rho(x) = int f dv (Sec. 2, Eq. (vlasov-poisson)) by the   */
/* tensor Gauss-Legendre rule in v: weight (h_v1 w_j3)(h_v2 w_j4).           */
/* ------------------------------------------------------------------------ */
int orc_rho(const orc_grid* g, const double* f, double* rho) {
  int n = g->deg + 1;
  double xi[ORC_MAXN], w[ORC_MAXN];
  long D[4], S[4];
  orc_gauss_legendre(n, xi, w);
  strides(g, D, S);
  long Dx = D[0] * D[1];
#pragma omp parallel for schedule(static)
  for (long p = 0; p < Dx; ++p) {
    ksum k = {0.0, 0.0};
    for (long i3 = 0; i3 < D[3]; ++i3)
      for (long i2 = 0; i2 < D[2]; ++i2)
        kadd(&k, node_weight(g, 2, i2, w) * node_weight(g, 3, i3, w) *
                     f[i3 * S[3] + i2 * S[2] + p]);
    rho[p] = kval(&k);
  }
  return 0;
}

/* The same v-quadrature for one x-node whose v-plane col[i3][i2] (D2*D3
   values, v1 fastest) was gathered out of f. */
double orc_rho_column(const orc_grid* g, const double* col) {
  int n = g->deg + 1;
  double xi[ORC_MAXN], w[ORC_MAXN];
  long D[4], S[4];
  orc_gauss_legendre(n, xi, w);
  strides(g, D, S);
  ksum k = {0.0, 0.0};
  for (long i3 = 0; i3 < D[3]; ++i3)
    for (long i2 = 0; i2 < D[2]; ++i2)
      kadd(&k, node_weight(g, 2, i2, w) * node_weight(g, 3, i3, w) * col[i3 * D[2] + i2]);
  return kval(&k);
}

/* lam[v][x] += (h_v1 w)(h_v2 w) rhobar[x]: the transpose of orc_rho. */
int orc_rho_adj(const orc_grid* g, const double* rhobar, double* lam) {
  int n = g->deg + 1;
  double xi[ORC_MAXN], w[ORC_MAXN];
  long D[4], S[4];
  orc_gauss_legendre(n, xi, w);
  strides(g, D, S);
  long Dx = D[0] * D[1];
#pragma omp parallel for schedule(static)
  for (long i3 = 0; i3 < D[3]; ++i3)
    for (long i2 = 0; i2 < D[2]; ++i2)
      for (long p = 0; p < Dx; ++p)
        lam[i3 * S[3] + i2 * S[2] + p] +=
            node_weight(g, 2, i2, w) * node_weight(g, 3, i3, w) * rhobar[p];
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Poisson map E = L rho (Sec. 3, the field solve is spectral; Eq.           */
/* (vlasov-poisson): div E = rho - 1, curl E = 0).  On the Gauss-Legendre   */
/* nodes z_n with weights w_n = h w_j the map is                             */
/*   rho_hat(m) = 1/(L1 L2) sum_n w_n1 w_n2 rho(n) exp(-i(k1 m1 z_n1 + k2 m2 z_n2)) */
/*   E_hat_d(m) = -i k_d m_d rho_hat(m) / (k1^2 m1^2 + k2^2 m2^2),  m != 0   */
/*   E_d(n)     = Re sum_{|m_d| <= K_d, m != 0} E_hat_d(m) exp(i(k.m.z_n))   */
/* with k_d = 2 pi / L_d.  The m = 0 mode is dropped, which removes the      */
/* constant background.  Default K_d = min(nc_d - 1, floor((D_d - 1)/2)).    */
/* The 2D sums are written as the matrix products                            */
/* F1 rho F2^T and G1 E_hat G2^T of the 1D transform matrices.               */
/* ------------------------------------------------------------------------ */
typedef struct {
  long D[2];
  int K[2];
  double kap[2];
  double complex* F[2]; /* (2K+1) x D: w_n exp(-i k m z_n) / L */
  double complex* G[2]; /* D x (2K+1): exp(i k m z_n) */
} orc_spec;

static void spec_init(const orc_grid* g, orc_spec* sp) {
  int n = g->deg + 1;
  double xi[ORC_MAXN], w[ORC_MAXN];
  orc_gauss_legendre(n, xi, w);
  for (int d = 0; d < 2; ++d) {
    long D = dimlen(g, d);
    double L = g->hi[d] - g->lo[d];
    /* default: modes |m| <= nc-1.  The composite Gauss-Legendre rule sums
       exp(i k j z) exactly to zero for 0 < |j| < nc but not at j = nc, so a
       mode |m| >= nc would pick up the constant background (aliasing). */
    int K = (int)((D - 1) / 2);
    if (K > g->nc[d] - 1) K = g->nc[d] - 1;
    if (g->kmax >= 0) K = g->kmax;
    sp->D[d] = D;
    sp->K[d] = K;
    sp->kap[d] = 2.0 * M_PI / L;
    long M = 2 * K + 1;
    sp->F[d] = (double complex*)malloc((size_t)(M * D) * sizeof(double complex));
    sp->G[d] = (double complex*)malloc((size_t)(M * D) * sizeof(double complex));
    for (long mi = 0; mi < M; ++mi) {
      double m = (double)(mi - K);
      for (long i = 0; i < D; ++i) {
        double z = node_coord(g, d, i, xi);
        double ph = sp->kap[d] * m * z;
        sp->F[d][mi * D + i] = node_weight(g, d, i, w) / L * (cos(ph) - I * sin(ph));
        sp->G[d][i * M + mi] = cos(ph) + I * sin(ph);
      }
    }
  }
}

static void spec_free(orc_spec* sp) {
  for (int d = 0; d < 2; ++d) { free(sp->F[d]); free(sp->G[d]); }
}

/* multiplier c_d(m) = -i k_d m_d / |k m|^2, zero at m = 0 */
static double complex spec_mult(const orc_spec* sp, int d, long m1, long m2) {
  if (m1 == 0 && m2 == 0) return 0.0;
  double k1 = sp->kap[0] * m1, k2 = sp->kap[1] * m2;
  double kd = d == 0 ? k1 : k2;
  return -I * kd / (k1 * k1 + k2 * k2);
}

int orc_poisson(const orc_grid* g, const double* rho, double* E1, double* E2) {
  orc_spec sp;
  spec_init(g, &sp);
  long D1 = sp.D[0], D2 = sp.D[1];
  long M1 = 2 * sp.K[0] + 1, M2 = 2 * sp.K[1] + 1;
  double complex* T = (double complex*)malloc((size_t)(D2 * M1) * sizeof(double complex));
  double complex* R = (double complex*)malloc((size_t)(M2 * M1) * sizeof(double complex));
  double complex* U = (double complex*)malloc((size_t)(D2 * M1) * sizeof(double complex));
  /* T[n2][m1] = sum_n1 F1[m1][n1] rho[n2][n1] */
  for (long n2 = 0; n2 < D2; ++n2)
    for (long m1 = 0; m1 < M1; ++m1) {
      double complex acc = 0.0;
      for (long n1 = 0; n1 < D1; ++n1) acc += sp.F[0][m1 * D1 + n1] * rho[n2 * D1 + n1];
      T[n2 * M1 + m1] = acc;
    }
  /* R[m2][m1] = sum_n2 F2[m2][n2] T[n2][m1] = rho_hat(m1, m2) */
  for (long m2 = 0; m2 < M2; ++m2)
    for (long m1 = 0; m1 < M1; ++m1) {
      double complex acc = 0.0;
      for (long n2 = 0; n2 < D2; ++n2) acc += sp.F[1][m2 * D2 + n2] * T[n2 * M1 + m1];
      R[m2 * M1 + m1] = acc;
    }
  for (int d = 0; d < 2; ++d) {
    double* E = d == 0 ? E1 : E2;
    /* U[n2][m1] = sum_m2 G2[n2][m2] c_d(m) rho_hat(m) */
    for (long n2 = 0; n2 < D2; ++n2)
      for (long m1 = 0; m1 < M1; ++m1) {
        double complex acc = 0.0;
        for (long m2 = 0; m2 < M2; ++m2)
          acc += sp.G[1][n2 * M2 + m2] * spec_mult(&sp, d, m1 - sp.K[0], m2 - sp.K[1]) *
                 R[m2 * M1 + m1];
        U[n2 * M1 + m1] = acc;
      }
    /* E[n2][n1] = Re sum_m1 G1[n1][m1] U[n2][m1] */
    for (long n2 = 0; n2 < D2; ++n2)
      for (long n1 = 0; n1 < D1; ++n1) {
        double complex acc = 0.0;
        for (long m1 = 0; m1 < M1; ++m1) acc += sp.G[0][n1 * M1 + m1] * U[n2 * M1 + m1];
        E[n2 * D1 + n1] = creal(acc);
      }
  }
  free(T);
  free(R);
  free(U);
  spec_free(&sp);
  return 0;
}

/* Transpose of the real-linear map rho -> (E1, E2):                         */
/*   rhobar = Re F1^T ( sum_d c_d .* (G1^T Ebar_d G2) ) F2                   */
int orc_poisson_adj(const orc_grid* g, const double* E1bar, const double* E2bar,
                    double* rhobar) {
  orc_spec sp;
  spec_init(g, &sp);
  long D1 = sp.D[0], D2 = sp.D[1];
  long M1 = 2 * sp.K[0] + 1, M2 = 2 * sp.K[1] + 1;
  double complex* V = (double complex*)malloc((size_t)(D2 * M1) * sizeof(double complex));
  double complex* P = (double complex*)calloc((size_t)(M2 * M1), sizeof(double complex));
  double complex* Y = (double complex*)malloc((size_t)(D2 * M1) * sizeof(double complex));
  for (int d = 0; d < 2; ++d) {
    const double* Eb = d == 0 ? E1bar : E2bar;
    /* V[n2][m1] = sum_n1 G1[n1][m1] Ebar[n2][n1] */
    for (long n2 = 0; n2 < D2; ++n2)
      for (long m1 = 0; m1 < M1; ++m1) {
        double complex acc = 0.0;
        for (long n1 = 0; n1 < D1; ++n1) acc += sp.G[0][n1 * M1 + m1] * Eb[n2 * D1 + n1];
        V[n2 * M1 + m1] = acc;
      }
    /* P[m2][m1] += c_d(m) sum_n2 G2[n2][m2] V[n2][m1] */
    for (long m2 = 0; m2 < M2; ++m2)
      for (long m1 = 0; m1 < M1; ++m1) {
        double complex acc = 0.0;
        for (long n2 = 0; n2 < D2; ++n2) acc += sp.G[1][n2 * M2 + m2] * V[n2 * M1 + m1];
        P[m2 * M1 + m1] += spec_mult(&sp, d, m1 - sp.K[0], m2 - sp.K[1]) * acc;
      }
  }
  /* Y[p2][m1] = sum_m2 F2[m2][p2] P[m2][m1] */
  for (long p2 = 0; p2 < D2; ++p2)
    for (long m1 = 0; m1 < M1; ++m1) {
      double complex acc = 0.0;
      for (long m2 = 0; m2 < M2; ++m2) acc += sp.F[1][m2 * D2 + p2] * P[m2 * M1 + m1];
      Y[p2 * M1 + m1] = acc;
    }
  /* rhobar[p2][p1] = Re sum_m1 F1[m1][p1] Y[p2][m1] */
  for (long p2 = 0; p2 < D2; ++p2)
    for (long p1 = 0; p1 < D1; ++p1) {
      double complex acc = 0.0;
      for (long m1 = 0; m1 < M1; ++m1) acc += sp.F[0][m1 * D1 + p1] * Y[p2 * M1 + m1];
      rhobar[p2 * D1 + p1] = creal(acc);
    }
  free(V);
  free(P);
  free(Y);
  spec_free(&sp);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Electric energy W = 1/2 sum_x w_x1 w_x2 (E1^2 + E2^2) (Sec. 4, Fig. 4:    */
/* "electric energy"; the factor 1/2 is this oracle's reading).              */
/* ------------------------------------------------------------------------ */
double orc_electric_energy(const orc_grid* g, const double* E1, const double* E2) {
  int n = g->deg + 1;
  double xi[ORC_MAXN], w[ORC_MAXN];
  orc_gauss_legendre(n, xi, w);
  long D0 = dimlen(g, 0), D1 = dimlen(g, 1);
  ksum k = {0.0, 0.0};
  for (long i1 = 0; i1 < D1; ++i1)
    for (long i0 = 0; i0 < D0; ++i0) {
      double e1 = E1[i1 * D0 + i0], e2 = E2[i1 * D0 + i0];
      kadd(&k, 0.5 * node_weight(g, 0, i0, w) * node_weight(g, 1, i1, w) * (e1 * e1 + e2 * e2));
    }
  return kval(&k);
}

/* ------------------------------------------------------------------------ */
/* Diagnostics (Sec. 4, Fig. 4; Sec. 5, Fig. 5): with the 4D tensor          */
/* Gauss-Legendre weight w,                                                  */
/*   out[0] mass   = sum w f                                                 */
/*   out[1] L1     = sum w |f|                                               */
/*   out[2] L2sq   = sum w f^2                                               */
/*   out[3] kinetic= 1/2 sum w (v1^2 + v2^2) f                               */
/*   out[4] W      = electric energy of (E1, E2)                             */
/*   out[5] total  = kinetic + W                                             */
/* ------------------------------------------------------------------------ */
int orc_diagnostics(const orc_grid* g, const double* f, const double* E1, const double* E2,
                    double* out) {
  int n = g->deg + 1;
  double xi[ORC_MAXN], w[ORC_MAXN];
  long D[4], S[4];
  orc_gauss_legendre(n, xi, w);
  strides(g, D, S);
  ksum km = {0, 0}, k1 = {0, 0}, k2 = {0, 0}, kk = {0, 0};
  for (long i3 = 0; i3 < D[3]; ++i3)
    for (long i2 = 0; i2 < D[2]; ++i2) {
      double v1 = node_coord(g, 2, i2, xi), v2 = node_coord(g, 3, i3, xi);
      double wv = node_weight(g, 2, i2, w) * node_weight(g, 3, i3, w);
      for (long i1 = 0; i1 < D[1]; ++i1)
        for (long i0 = 0; i0 < D[0]; ++i0) {
          double wt = node_weight(g, 0, i0, w) * node_weight(g, 1, i1, w) * wv;
          double x = f[i3 * S[3] + i2 * S[2] + i1 * S[1] + i0];
          kadd(&km, wt * x);
          kadd(&k1, wt * fabs(x));
          kadd(&k2, wt * x * x);
          kadd(&kk, 0.5 * wt * (v1 * v1 + v2 * v2) * x);
        }
    }
  out[0] = kval(&km);
  out[1] = kval(&k1);
  out[2] = kval(&k2);
  out[3] = kval(&kk);
  out[4] = (E1 && E2) ? orc_electric_energy(g, E1, E2) : 0.0;
  out[5] = out[3] + out[4];
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Initial values, evaluated at the nodes (nodal interpolation).             */
/*   kind 0, Landau (Sec. 4, Eq. (iv-nl)), params (eps, k1, k2):             */
/*     (1 + eps (cos k1 x1 + cos k2 x2)) exp(-(v1^2+v2^2)/2) / (2 pi)        */
/*   kind 1, two-stream, additive perturbation, params (eps, k, v0):         */
/*     (exp(-(v1-v0)^2/2) + exp(-(v1+v0)^2/2)) exp(-v2^2/2) / (4 pi)         */
/*       * (1 + eps cos k x1 + eps cos k x2)                                 */
/*   kind 2, two-stream of Sec. 5, Eq. (iv-tsi), params (eps, k, v0):        */
/*     (1 + eps cos k x1 cos k x2) (1/(8 pi)) (e^{-(v1-v0)^2/2}+e^{-(v1+v0)^2/2}) */
/*       (e^{-(v2-v0)^2/2}+e^{-(v2+v0)^2/2})                                 */
/* ------------------------------------------------------------------------ */
int orc_init(const orc_grid* g, int kind, const double* p, double* f) {
  int n = g->deg + 1;
  double xi[ORC_MAXN], w[ORC_MAXN];
  long D[4], S[4];
  if (kind < 0 || kind > 2) return -1;
  orc_gauss_legendre(n, xi, w);
  strides(g, D, S);
#pragma omp parallel for schedule(static)
  for (long i3 = 0; i3 < D[3]; ++i3)
    for (long i2 = 0; i2 < D[2]; ++i2)
      for (long i1 = 0; i1 < D[1]; ++i1)
        for (long i0 = 0; i0 < D[0]; ++i0) {
          double x1 = node_coord(g, 0, i0, xi), x2 = node_coord(g, 1, i1, xi);
          double v1 = node_coord(g, 2, i2, xi), v2 = node_coord(g, 3, i3, xi);
          double val;
          if (kind == 0) {
            val = (1.0 + p[0] * (cos(p[1] * x1) + cos(p[2] * x2))) *
                  exp(-(v1 * v1 + v2 * v2) / 2.0) / (2.0 * M_PI);
          } else if (kind == 1) {
            val = (exp(-(v1 - p[2]) * (v1 - p[2]) / 2.0) + exp(-(v1 + p[2]) * (v1 + p[2]) / 2.0)) *
                  exp(-v2 * v2 / 2.0) / (4.0 * M_PI) *
                  (1.0 + p[0] * cos(p[1] * x1) + p[0] * cos(p[1] * x2));
          } else {
            val = (1.0 + p[0] * cos(p[1] * x1) * cos(p[1] * x2)) / (8.0 * M_PI) *
                  (exp(-(v1 - p[2]) * (v1 - p[2]) / 2.0) + exp(-(v1 + p[2]) * (v1 + p[2]) / 2.0)) *
                  (exp(-(v2 - p[2]) * (v2 - p[2]) / 2.0) + exp(-(v2 + p[2]) * (v2 + p[2]) / 2.0));
          }
          f[i3 * S[3] + i2 * S[2] + i1 * S[1] + i0] = val;
        }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Strang step (Sec. 2): f^{m+1} = e^{tau/2 A} e^{tau B} e^{tau/2 A} f^m,    */
/* with e^{tau A} = e^{tau A2} e^{tau A1} and the kick split into v1 then   */
/* v2, E frozen at the rho after the first half drift.                       */
/*   g1 = X1(tau/2) f; g2 = X2(tau/2) g1; rho = Q g2; E = L rho;             */
/*   g3 = V1(tau E1) g2; g4 = V2(tau E2) g3; g5 = X1(tau/2) g4;              */
/*   f^{m+1} = X2(tau/2) g5.                                                 */
/* kick = 0 replaces E by zero (free streaming).  W_hist[m] = W(E^m).        */
/* E1, E2 (nullable) receive the last step's field.                          */
/* ------------------------------------------------------------------------ */
typedef struct {
  double *rho, *E1, *E2;
} orc_fields;

static void step_once(const orc_grid* g, double* f, double* tmp, int kick, orc_fields* fl,
                      double* Wout) {
  long Dx = dimlen(g, 0) * dimlen(g, 1);
  orc_sweep(g, 0, NULL, 0.5, f, tmp);
  orc_sweep(g, 1, NULL, 0.5, tmp, f);
  if (kick) {
    orc_rho(g, f, fl->rho);
    orc_poisson(g, fl->rho, fl->E1, fl->E2);
  } else {
    for (long p = 0; p < Dx; ++p) fl->E1[p] = fl->E2[p] = 0.0;
  }
  if (Wout) *Wout = orc_electric_energy(g, fl->E1, fl->E2);
  orc_sweep(g, 2, fl->E1, 1.0, f, tmp);
  orc_sweep(g, 3, fl->E2, 1.0, tmp, f);
  orc_sweep(g, 0, NULL, 0.5, f, tmp);
  orc_sweep(g, 1, NULL, 0.5, tmp, f);
}

int orc_step(const orc_grid* g, double* f, int nsteps, int kick, double* W_hist, double* E1,
             double* E2) {
  long N = orc_numel(g), Dx = dimlen(g, 0) * dimlen(g, 1);
  double* tmp = (double*)malloc((size_t)N * sizeof(double));
  orc_fields fl;
  fl.rho = (double*)malloc((size_t)Dx * sizeof(double));
  fl.E1 = (double*)malloc((size_t)Dx * sizeof(double));
  fl.E2 = (double*)malloc((size_t)Dx * sizeof(double));
  if (!tmp || !fl.rho || !fl.E1 || !fl.E2) return -3;
  for (int m = 0; m < nsteps; ++m) step_once(g, f, tmp, kick, &fl, W_hist ? &W_hist[m] : NULL);
  if (E1) memcpy(E1, fl.E1, (size_t)Dx * sizeof(double));
  if (E2) memcpy(E2, fl.E2, (size_t)Dx * sizeof(double));
  free(tmp);
  free(fl.rho);
  free(fl.E1);
  free(fl.E2);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Splitting compositions built on the Strang step (Sec. 2 cites higher     */
/* order splittings).  order 2: the Strang step itself.  order 4: the       */
/* symmetric triple jump S(g1 tau) S(g0 tau) S(g1 tau) of Strang steps,     */
/* g1 = 1 / (2 - 2^(1/3)), g0 = 1 - 2 g1 (g0 < 0): the weights with         */
/* 2 g1 + g0 = 1 and 2 g1^3 + g0^3 = 0, which cancel the tau^3 error of a   */
/* symmetric second-order step.                                             */
/* Stage list of nsteps steps: kind 0 = drift e^{frac tau A} (x1 then x2),  */
/* 1 = kick e^{frac tau B} (field from the current rho, v1 then v2), 2 = the */
/* first kick of a step (its W is recorded).  merge: consecutive drifts     */
/* (across sub-steps and steps) become one drift of the summed fraction,    */
/* which equals the separate drifts for the exact flow but not after the    */
/* SLDG projection.  Returns the number of stages, -1 if cap is too small   */
/* or the order is not 2 or 4.                                              */
/* ------------------------------------------------------------------------ */
static int push_stage(int* kind, double* frac, int* n, int cap, int k, double fr) {
  if (*n >= cap) return -1;
  kind[*n] = k;
  frac[*n] = fr;
  ++*n;
  return 0;
}

int orc_split_stages(int order, int nsteps, int merge, int* kind, double* frac, int cap) {
  double gam[3];
  int ns;
  if (order == 2) {
    gam[0] = 1.0;
    ns = 1;
  } else if (order == 4) {
    gam[0] = 1.0 / (2.0 - cbrt(2.0));
    gam[1] = 1.0 - 2.0 * gam[0];
    gam[2] = gam[0];
    ns = 3;
  } else {
    return -1;
  }
  int n = 0;
  double pending = 0.0; /* merge: the drift carried over from the last kick */
  for (int m = 0; m < nsteps; ++m)
    for (int i = 0; i < ns; ++i) {
      const double a = 0.5 * gam[i];
      if (push_stage(kind, frac, &n, cap, 0, merge ? pending + a : a)) return -1;
      if (push_stage(kind, frac, &n, cap, i == 0 ? 2 : 1, gam[i])) return -1;
      if (merge)
        pending = a;
      else if (push_stage(kind, frac, &n, cap, 0, a))
        return -1;
    }
  if (merge && nsteps > 0 && push_stage(kind, frac, &n, cap, 0, pending)) return -1;
  return n;
}

/* nsteps steps of the composition (order, merge) of orc_split_stages; the
 * arguments and outputs as orc_step (W_hist[m]: W at the first kick of step
 * m). */
int orc_step_split(const orc_grid* g, double* f, int nsteps, int order, int merge, int kick,
                   double* W_hist, double* E1, double* E2) {
  const int cap = 9 * nsteps + 2;
  int* kind = (int*)malloc((size_t)cap * sizeof(int));
  double* fr = (double*)malloc((size_t)cap * sizeof(double));
  long N = orc_numel(g), Dx = dimlen(g, 0) * dimlen(g, 1);
  double* tmp = (double*)malloc((size_t)N * sizeof(double));
  orc_fields fl;
  fl.rho = (double*)malloc((size_t)Dx * sizeof(double));
  fl.E1 = (double*)calloc((size_t)Dx, sizeof(double));
  fl.E2 = (double*)calloc((size_t)Dx, sizeof(double));
  if (!kind || !fr || !tmp || !fl.rho || !fl.E1 || !fl.E2) return -3;
  const int n = orc_split_stages(order, nsteps, merge, kind, fr, cap);
  if (n < 0) return -1;
  int m = 0;
  for (int q = 0; q < n; ++q) {
    if (kind[q] == 0) {
      orc_sweep(g, 0, NULL, fr[q], f, tmp);
      orc_sweep(g, 1, NULL, fr[q], tmp, f);
      continue;
    }
    if (kick) {
      orc_rho(g, f, fl.rho);
      orc_poisson(g, fl.rho, fl.E1, fl.E2);
    } else {
      for (long p = 0; p < Dx; ++p) fl.E1[p] = fl.E2[p] = 0.0;
    }
    if (kind[q] == 2) {
      if (W_hist) W_hist[m] = orc_electric_energy(g, fl.E1, fl.E2);
      ++m;
    }
    orc_sweep(g, 2, fl.E1, fr[q], f, tmp);
    orc_sweep(g, 3, fl.E2, fr[q], tmp, f);
  }
  if (E1) memcpy(E1, fl.E1, (size_t)Dx * sizeof(double));
  if (E2) memcpy(E2, fl.E2, (size_t)Dx * sizeof(double));
  free(kind);
  free(fr);
  free(tmp);
  free(fl.rho);
  free(fl.E1);
  free(fl.E2);
  return 0;
}

/* rho and E of the current f (no sweep). */
int orc_fields_of(const orc_grid* g, const double* f, double* rho, double* E1, double* E2) {
  orc_rho(g, f, rho);
  orc_poisson(g, rho, E1, E2);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Adjoint (reverse mode) of J = sum_m cW[m] W(E^m), the time-integrated     */
/* electric energy when cW[m] = tau (the default when cW is NULL).           */
/* grad = dJ/df^0 per stored nodal value.  Checkpoints f every ckpt steps;   */
/* each segment is recomputed forward, then walked in reverse:               */
/*   lam5 = X2^T lam; lam4 = X1^T lam5;                                      */
/*   lam3 = V2^T lam4, E2bar += d/dE2 <lam4, V2 g3>;                         */
/*   lam2 = V1^T lam3, E1bar += d/dE1 <lam3, V1 g2>;                         */
/*   Ebar += cW[m] w_x E;  rhobar = L^T Ebar;  lam2 += Q^T rhobar;           */
/*   lam1 = X2^T lam2; lam0 = X1^T lam1.                                     */
/* ------------------------------------------------------------------------ */
int orc_backward(const orc_grid* g, const double* f0, int nsteps, int ckpt, const double* cW,
                 double* grad, double* J_out, double* W_hist) {
  int n = g->deg + 1;
  double xi[ORC_MAXN], w[ORC_MAXN];
  orc_gauss_legendre(n, xi, w);
  long N = orc_numel(g), D0 = dimlen(g, 0), D1 = dimlen(g, 1), Dx = D0 * D1;
  if (ckpt < 1) ckpt = 1;
  int nck = (nsteps + ckpt - 1) / ckpt;
  if (nck < 1) nck = 1;
  double* cks = (double*)malloc((size_t)nck * (size_t)N * sizeof(double));
  double* seg = (double*)malloc((size_t)(ckpt + 1) * (size_t)N * sizeof(double));
  double* tmp = (double*)malloc((size_t)N * sizeof(double));
  double* g2 = (double*)malloc((size_t)N * sizeof(double));
  double* g3 = (double*)malloc((size_t)N * sizeof(double));
  double* lam = (double*)calloc((size_t)N, sizeof(double));
  double* lb = (double*)malloc((size_t)N * sizeof(double));
  double* rho = (double*)malloc((size_t)Dx * sizeof(double));
  double* E1 = (double*)malloc((size_t)Dx * sizeof(double));
  double* E2 = (double*)malloc((size_t)Dx * sizeof(double));
  double* Eb1 = (double*)malloc((size_t)Dx * sizeof(double));
  double* Eb2 = (double*)malloc((size_t)Dx * sizeof(double));
  double* rb = (double*)malloc((size_t)Dx * sizeof(double));
  if (!cks || !seg || !tmp || !g2 || !g3 || !lam || !lb || !rho || !E1 || !E2 || !Eb1 ||
      !Eb2 || !rb)
    return -3;
  orc_fields fl = {rho, E1, E2};
  /* forward pass: checkpoints and J */
  ksum kj = {0, 0};
  memcpy(tmp, f0, (size_t)N * sizeof(double));
  double* cur = g2; /* reuse as the running state */
  memcpy(cur, f0, (size_t)N * sizeof(double));
  for (int m = 0; m < nsteps; ++m) {
    if (m % ckpt == 0) memcpy(cks + (size_t)(m / ckpt) * N, cur, (size_t)N * sizeof(double));
    double Wm;
    step_once(g, cur, tmp, 1, &fl, &Wm);
    if (W_hist) W_hist[m] = Wm;
    kadd(&kj, (cW ? cW[m] : g->dt) * Wm);
  }
  if (J_out) *J_out = kval(&kj);
  /* reverse pass */
  for (int c = nck - 1; c >= 0; --c) {
    int m0 = c * ckpt, m1 = m0 + ckpt < nsteps ? m0 + ckpt : nsteps;
    memcpy(seg, cks + (size_t)c * N, (size_t)N * sizeof(double));
    for (int m = m0; m < m1 - 1; ++m) {
      double* nxt = seg + (size_t)(m - m0 + 1) * N;
      memcpy(nxt, seg + (size_t)(m - m0) * N, (size_t)N * sizeof(double));
      step_once(g, nxt, tmp, 1, &fl, NULL);
    }
    for (int m = m1 - 1; m >= m0; --m) {
      const double* fm = seg + (size_t)(m - m0) * N;
      /* recompute the forward intermediates g2 (before V1), g3 (before V2) */
      orc_sweep(g, 0, NULL, 0.5, fm, tmp);
      orc_sweep(g, 1, NULL, 0.5, tmp, g2);
      orc_rho(g, g2, rho);
      orc_poisson(g, rho, E1, E2);
      orc_sweep(g, 2, E1, 1.0, g2, g3);
      /* reverse */
      for (long p = 0; p < Dx; ++p) Eb1[p] = Eb2[p] = 0.0;
      orc_sweep_adj(g, 1, NULL, 0.5, lam, lb, NULL, NULL);   /* lam5 */
      orc_sweep_adj(g, 0, NULL, 0.5, lb, lam, NULL, NULL);   /* lam4 */
      orc_sweep_adj(g, 3, E2, 1.0, lam, lb, g3, Eb2);        /* lam3 */
      orc_sweep_adj(g, 2, E1, 1.0, lb, lam, g2, Eb1);        /* lam2 */
      double cm = cW ? cW[m] : g->dt;
      for (long i1 = 0; i1 < D1; ++i1)
        for (long i0 = 0; i0 < D0; ++i0) {
          double wx = node_weight(g, 0, i0, w) * node_weight(g, 1, i1, w);
          Eb1[i1 * D0 + i0] += cm * wx * E1[i1 * D0 + i0];
          Eb2[i1 * D0 + i0] += cm * wx * E2[i1 * D0 + i0];
        }
      orc_poisson_adj(g, Eb1, Eb2, rb);
      orc_rho_adj(g, rb, lam);
      orc_sweep_adj(g, 1, NULL, 0.5, lam, lb, NULL, NULL);   /* lam1 */
      orc_sweep_adj(g, 0, NULL, 0.5, lb, lam, NULL, NULL);   /* lam0 */
    }
  }
  memcpy(grad, lam, (size_t)N * sizeof(double));
  free(cks); free(seg); free(tmp); free(g2); free(g3); free(lam); free(lb);
  free(rho); free(E1); free(E2); free(Eb1); free(Eb2); free(rb);
  return 0;
}

/* Number of threads the oracle's parallel loops use (1 without OpenMP). */
#ifdef _OPENMP
#include <omp.h>
int orc_threads(void) { return omp_get_max_threads(); }
#else
int orc_threads(void) { return 1; }
#endif
