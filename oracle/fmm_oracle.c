/*
 * oracle/fmm_oracle.c -- TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT PATH.
 *
 * A plain, slow, FP64 CPU restatement of the method of Ibeid, Yokota, Pestana and
 * Keyes, "Fast Multipole Preconditioners for Sparse Matrices Arising from Elliptic
 * Equations" (arXiv:1308.3339): a finite-difference Poisson system solved by a Krylov
 * method whose preconditioner is a free-space Laplace FMM over the grid nodes plus a
 * boundary-element correction (Sec. 3.2, Fig. f:flow_chart).
 *
 * Only tests/, __graft_entry__.smoke() and the CPU legs of bench.py load this file.
 * It shares no code, header, table or constant generator with the CUDA library, and
 * it never imports or calls it.  Every routine follows one passage of the paper, in
 * the paper's notation and order, with no blocking or fusion beyond what the passage
 * states.  Where the paper is silent the reading taken is stated at the routine.
 *
 * Units: physical coordinates throughout.  Domain [x0, x0+side]^2, n interior nodes per
 * side, h = side/(n+1), node (i,j) (0-based) at (x0+(i+1)h, y0+(j+1)h), natural index
 * j*n+i.  Expansions are the unscaled complex coefficients M_n, L_n of Sec. 5.3.
 *
 * Parity status: every function below is pinned by a CPU test (closed forms,
 * quadrature, brute force, FFT lattice sums, exactness identities); none is
 * "parity unpinned".
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;
static const double PI_ = 3.14159265358979323846264338327950288;

int orc_version(void) { return 3; }

int orc_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ======================================================================== */
/* 1. Discrete system (Sec. 2.1, Eq. e:p with a = 1, Eq. e:axb).             */
/*    The paper discretises with Q1 elements; the workload here is the       */
/*    5-point finite-difference stencil, A = (1/h^2)(4u_ij - neighbours).     */
/* ======================================================================== */

/* y = A x with zero Dirichlet values outside the n x n interior block. */
void orc_spmv5(int n, double h, const double *x, double *y) {
  const double s = 1.0 / (h * h);
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) {
      double v = 4.0 * x[j * n + i];
      if (i > 0) v -= x[j * n + i - 1];
      if (i < n - 1) v -= x[j * n + i + 1];
      if (j > 0) v -= x[(j - 1) * n + i];
      if (j < n - 1) v -= x[(j + 1) * n + i];
      y[j * n + i] = s * v;
    }
}

/* b = f + (1/h^2) * g at the boundary neighbours (Eq. e:pbound moved to the right-hand
 * side of e:axb).  g holds 4n values: bottom (x increasing), right (y increasing),
 * top (x decreasing), left (y decreasing); corners are never referenced. */
void orc_fold_rhs(int n, double h, const double *f, const double *g, double *b) {
  const double s = 1.0 / (h * h);
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) {
      double v = f[j * n + i];
      if (g) {
        if (j == 0) v += s * g[i];
        if (i == n - 1) v += s * g[n + j];
        if (j == n - 1) v += s * g[2 * n + (n - 1 - i)];
        if (i == 0) v += s * g[3 * n + (n - 1 - j)];
      }
      b[j * n + i] = v;
    }
}

/* ======================================================================== */
/* 1b. Variable diffusion coefficient (Sec. 4.4; the problem of Sec. 6.4,    */
/*     -div(a grad u) = f with a = 1 + mu sin(m pi x) sin(n pi y)).          */
/*     Five-point flux form: the coefficient of the face between two nodes   */
/*     is the mean of a at the two nodes; a is given at the (n+2)^2 nodes of  */
/*     the full grid, boundary ring included, row-major, node (i, j) of the   */
/*     interior at full index (j+1)(n+2) + (i+1).                             */
/* ======================================================================== */

void orc_spmv5_var(int n, double h, const double *a, const double *x, double *y) {
  const double s = 1.0 / (h * h);
  const int W = n + 2;
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) {
      const int ic = (j + 1) * W + (i + 1);
      const double aE = 0.5 * (a[ic] + a[ic + 1]), aW = 0.5 * (a[ic] + a[ic - 1]);
      const double aN = 0.5 * (a[ic] + a[ic + W]), aS = 0.5 * (a[ic] + a[ic - W]);
      double v = (aE + aW + aN + aS) * x[j * n + i];
      if (i > 0) v -= aW * x[j * n + i - 1];
      if (i < n - 1) v -= aE * x[j * n + i + 1];
      if (j > 0) v -= aS * x[(j - 1) * n + i];
      if (j < n - 1) v -= aN * x[(j + 1) * n + i];
      y[j * n + i] = s * v;
    }
}

/* b = f + (1/h^2) a_face g at the boundary neighbours (layout of g as in orc_fold_rhs). */
void orc_fold_rhs_var(int n, double h, const double *a, const double *f, const double *g, double *b) {
  const double s = 1.0 / (h * h);
  const int W = n + 2;
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) {
      const int ic = (j + 1) * W + (i + 1);
      double v = f[j * n + i];
      if (g) {
        if (j == 0) v += s * 0.5 * (a[ic] + a[ic - W]) * g[i];
        if (i == n - 1) v += s * 0.5 * (a[ic] + a[ic + 1]) * g[n + j];
        if (j == n - 1) v += s * 0.5 * (a[ic] + a[ic + W]) * g[2 * n + (n - 1 - i)];
        if (i == 0) v += s * 0.5 * (a[ic] + a[ic - 1]) * g[3 * n + (n - 1 - j)];
      }
      b[j * n + i] = v;
    }
}

/* ======================================================================== */
/* 1c. Q1 bilinear finite elements, the paper's discretisation (Sec. 6.1),   */
/*     on the uniform square grid with zero Dirichlet values: the stiffness   */
/*     of -lap sums the element integrals of grad phi_i . grad phi_j over the */
/*     four elements around node i, giving 8/3 on the diagonal and -1/3 for   */
/*     each of the eight neighbours (independent of h in two dimensions).     */
/*     Load vector: the lumped Q1 mass, b_i = h^2 f_i (exact for the constant */
/*     f of Table t:p1).                                                      */
/* ======================================================================== */

void orc_spmv_q1(int n, const double *x, double *y) {
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) {
      double v = (8.0 / 3.0) * x[j * n + i];
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          if (dx == 0 && dy == 0) continue;
          const int ii = i + dx, jj = j + dy;
          if (ii < 0 || ii >= n || jj < 0 || jj >= n) continue;
          v -= (1.0 / 3.0) * x[jj * n + ii];
        }
      y[j * n + i] = v;
    }
}

void orc_q1_load(int n, double h, const double *f, double *b) {
  for (int k = 0; k < n * n; ++k) b[k] = h * h * f[k];
}

/* The FMM-BEM preconditioner inverts the continuous operator, so on a Q1 residual r (a
 * functional, r_i = int r phi_i) it acts on the finite-element function whose coefficients
 * solve M c = r, M the consistent Q1 mass matrix of the interior nodes.  On the uniform grid
 * M = h^2 (M1 (x) M1) with M1 = tridiag(1, 4, 1)/6, so c follows from tridiagonal solves
 * along every row and then every column (Thomas algorithm). */
static void tridiag_141_solve(int n, double *x, int stride, double *cp) {
  /* (1/6) tridiag(1, 4, 1) y = x, in place, elements x[k stride] */
  double prev = 0.0;
  for (int k = 0; k < n; ++k) {
    const double den = 4.0 / 6.0 - (k ? (1.0 / 6.0) * cp[k - 1] : 0.0);
    cp[k] = (1.0 / 6.0) / den;
    prev = (x[(int64_t)k * stride] - (k ? (1.0 / 6.0) * prev : 0.0)) / den;
    x[(int64_t)k * stride] = prev;
  }
  for (int k = n - 2; k >= 0; --k) x[(int64_t)k * stride] -= cp[k] * x[(int64_t)(k + 1) * stride];
}

void orc_q1_mass_solve(int n, double h, const double *r, double *c) {
  double *cp = malloc(sizeof(double) * n);
  for (int k = 0; k < n * n; ++k) c[k] = r[k] / (h * h);
  for (int j = 0; j < n; ++j) tridiag_141_solve(n, c + (int64_t)j * n, 1, cp);  /* rows */
  for (int i = 0; i < n; ++i) tridiag_141_solve(n, c + i, n, cp);              /* columns */
  free(cp);
}

/* ======================================================================== */
/* 2. Green's function and the volume operator (Sec. 4.2 Eq. eq:green,       */
/*    Sec. 5.1 Eq. e:volume_integral).                                        */
/*    (V r)_i = sum_j h^2 r_j G_ij,  G_ij = -(1/2pi) ln|x_i - x_j|.           */
/*    Reading for the singular i == j term (the paper smooths G with an       */
/*    unstated epsilon): G_ii is the mean of G over the node's h x h cell,     */
/*    -(1/2pi)(ln h + C_SELF) with C_SELF = mean of ln|x| over the unit       */
/*    square centred at 0 = -(ln 2)/2 - 3/2 + pi/4, from the closed form       */
/*    int_0^a int_0^a ln(x^2+y^2) = a^2 (ln(2a^2) - 3 + pi/2).                */
/* ======================================================================== */

double orc_self_constant(void) { return -0.5 * log(2.0) - 1.5 + 0.25 * PI_; }

/* ln|x_i - x_j| for nodes, with the cell-mean value on the diagonal. */
static double node_log(double h, double xi, double yi, double xj, double yj, int same) {
  if (same) return log(h) + orc_self_constant();
  double dx = xi - xj, dy = yi - yj;
  return 0.5 * log(dx * dx + dy * dy);
}

/* Direct O(N^2) sum of Eq. e:volume_integral at every node: out_i = (V r)_i. */
void orc_direct_V(int n, double x0, double y0, double side, const double *r, double *out) {
  const double h = side / (n + 1);
  const int N = n * n;
#pragma omp parallel for schedule(dynamic, 16)
  for (int t = 0; t < N; ++t) {
    double xi = x0 + (t % n + 1) * h, yi = y0 + (t / n + 1) * h, acc = 0.0;
    for (int s = 0; s < N; ++s) {
      double xj = x0 + (s % n + 1) * h, yj = y0 + (s / n + 1) * h;
      acc += h * h * r[s] * node_log(h, xi, yi, xj, yj, s == t);
    }
    out[t] = -acc / (2.0 * PI_);
  }
}

/* Direct sum at arbitrary targets that never coincide with a node. */
void orc_direct_V_at(int n, double x0, double y0, double side, const double *r, int nt,
                     const double *tx, const double *ty, double *out) {
  const double h = side / (n + 1);
  const int N = n * n;
#pragma omp parallel for schedule(dynamic, 16)
  for (int t = 0; t < nt; ++t) {
    double acc = 0.0;
    for (int s = 0; s < N; ++s) {
      double dx = tx[t] - (x0 + (s % n + 1) * h), dy = ty[t] - (y0 + (s / n + 1) * h);
      acc += h * h * r[s] * 0.5 * log(dx * dx + dy * dy);
    }
    out[t] = -acc / (2.0 * PI_);
  }
}

/* Direct sum at a subset of nodes (natural indices idx[0..nt)). */
void orc_direct_V_nodes(int n, double x0, double y0, double side, const double *r, int nt,
                        const int32_t *idx, double *out) {
  const double h = side / (n + 1);
  const int N = n * n;
#pragma omp parallel for schedule(dynamic, 4)
  for (int q = 0; q < nt; ++q) {
    int t = idx[q];
    double xi = x0 + (t % n + 1) * h, yi = y0 + (t / n + 1) * h, acc = 0.0;
    for (int s = 0; s < N; ++s) {
      double xj = x0 + (s % n + 1) * h, yj = y0 + (s / n + 1) * h;
      acc += h * h * r[s] * node_log(h, xi, yi, xj, yj, s == t);
    }
    out[q] = -acc / (2.0 * PI_);
  }
}

/* ======================================================================== */
/* 3. Expansions (Sec. 5.3).  Coefficients n = 0..p-1 ("pth order            */
/*    truncation").  They represent phi(z) = sum_j f_j log(z - z_j); the     */
/*    potential is u = -(1/2pi) Re phi, the factor the L2P formula leaves      */
/*    out.  Notation z_ab = z_a - z_b as in Fig. f:vectors.                    */
/* ======================================================================== */

/* Binomial coefficients from Pascal's triangle (exact in FP64 for the orders used). */
#define ORC_PMAX 40
static double g_binom[2 * ORC_PMAX + 2][2 * ORC_PMAX + 2];
static int g_binom_ready = 0;
static void binom_init(void) {
  if (g_binom_ready) return;
  for (int a = 0; a < 2 * ORC_PMAX + 2; ++a)
    for (int b = 0; b < 2 * ORC_PMAX + 2; ++b)
      g_binom[a][b] = (b == 0) ? 1.0 : (a == 0 ? 0.0 : g_binom[a - 1][b - 1] + g_binom[a - 1][b]);
  g_binom_ready = 1;
}
static double binom(int a, int b) {
  if (b < 0 || b > a) return 0.0;
  return g_binom[a][b];
}

/* pw[k] = z^k for k = 0..K */
static void powers(cplx z, int K, cplx *pw) {
  pw[0] = 1.0;
  for (int k = 1; k <= K; ++k) pw[k] = pw[k - 1] * z;
}

static cplx ipow(cplx z, int k) {
  cplx r = 1.0;
  for (int i = 0; i < k; ++i) r *= z;
  return r;
}

/* P2M: M_0 = sum f_j ; M_n = sum -f_j (-z_muj)^n / n. Adds into M. */
void orc_p2m(int p, int np, const double *px, const double *py, const double *f, double cx,
             double cy, cplx *M) {
  const cplx zmu = cx + I * cy;
  cplx pw[ORC_PMAX + 1];
  for (int j = 0; j < np; ++j) {
    cplx zmuj = zmu - (px[j] + I * py[j]);
    powers(-zmuj, p, pw);
    M[0] += f[j];
    for (int k = 1; k < p; ++k) M[k] += -f[j] * pw[k] / k;
  }
}

/* M2M from child mu to parent M, zMmu = z_M - z_mu. Adds into Mp. */
static void m2m_(int p, const cplx *Mc, cplx zMmu, cplx *Mp) {
  cplx pw[ORC_PMAX + 1];
  binom_init();
  powers(-zMmu, p, pw);
  Mp[0] += Mc[0];
  for (int k = 1; k < p; ++k) {
    cplx v = -Mc[0] * pw[k] / k;
    for (int q = 1; q <= k; ++q) v += Mc[q] * pw[k - q] * binom(k - 1, q - 1);
    Mp[k] += v;
  }
}

/* M2L from multipole at z_M to local at z_Lambda, zLM = z_Lambda - z_M. Adds into L. */
static void m2l_(int p, const cplx *M, cplx zLM, cplx *L) {
  cplx inv[2 * ORC_PMAX + 1];
  binom_init();
  powers(1.0 / zLM, 2 * p, inv); /* inv[k] = 1 / zLM^k */
  cplx v = M[0] * clog(zLM);
  for (int k = 1; k < p; ++k) v += M[k] * inv[k];
  L[0] += v;
  for (int nn = 1; nn < p; ++nn) {
    double sgn = (nn % 2) ? -1.0 : 1.0; /* (-1)^n */
    cplx w = -M[0] * sgn * inv[nn] / nn; /* -M_0 / ((-z)^n n) */
    for (int k = 1; k < p; ++k) w += sgn * M[k] * inv[nn + k] * binom(nn + k - 1, k - 1);
    L[nn] += w;
  }
}

/* L2L from parent Lambda to child lambda, zlL = z_lambda - z_Lambda. Adds into Lc. */
static void l2l_(int p, const cplx *Lp, cplx zlL, cplx *Lc) {
  cplx pw[ORC_PMAX + 1];
  binom_init();
  powers(zlL, p, pw);
  for (int nn = 0; nn < p; ++nn) {
    cplx v = 0.0;
    for (int k = nn; k < p; ++k) v += Lp[k] * pw[k - nn] * binom(k, nn);
    Lc[nn] += v;
  }
}

/* L2P: Re sum_n L_n z_ilambda^n (without the -1/2pi factor). */
static double l2p_(int p, const cplx *L, cplx zil) {
  cplx v = 0.0, zp = 1.0;
  for (int nn = 0; nn < p; ++nn) { v += L[nn] * zp; zp *= zil; }
  return creal(v);
}

/* Direct evaluation of a multipole series at z (z_iM = z - z_M): Re(M_0 log z + sum M_k/z^k).
 * Not one of the paper's five kernels; used by the tests to check P2M and M2M alone. */
static double m2p_(int p, const cplx *M, cplx ziM) {
  cplx v = M[0] * clog(ziM);
  for (int k = 1; k < p; ++k) v += M[k] / ipow(ziM, k);
  return creal(v);
}

/* Exported forms of the translation kernels for the tests: the complex offset is passed
 * as two doubles (re, im). */
void orc_m2m(int p, const cplx *Mc, double zr, double zi, cplx *Mp) { m2m_(p, Mc, zr + I * zi, Mp); }
void orc_m2l(int p, const cplx *M, double zr, double zi, cplx *L) { m2l_(p, M, zr + I * zi, L); }
void orc_l2l(int p, const cplx *Lp, double zr, double zi, cplx *Lc) { l2l_(p, Lp, zr + I * zi, Lc); }
double orc_l2p(int p, const cplx *L, double zr, double zi) { return l2p_(p, L, zr + I * zi); }
double orc_m2p(int p, const cplx *M, double zr, double zi) { return m2p_(p, M, zr + I * zi); }

/* ======================================================================== */
/* 4. Boundary elements (Sec. 4.3): constant elements, no nodes at corners.  */
/*    Reading: each side of the square is cut into n equal elements          */
/*    (N_Gamma = 4n), collocation at element midpoints, traversal             */
/*    counter-clockwise (bottom, right, top, left), outward normal.           */
/*    Piecewise integrals of G and dG/dn over straight elements are done in   */
/*    closed form (Sec. 4.2 says analytic expressions exist).                  */
/* ======================================================================== */

/* int over segment [a,b] of ln|x - y| ds_y.  With s along the segment and d the
 * signed normal distance: F(s) = s ln sqrt(s^2+d^2) - s + d atan(s/d). */
static double segF(double s, double d) {
  if (d == 0.0) return (s == 0.0) ? 0.0 : s * log(fabs(s)) - s;
  return 0.5 * s * log(s * s + d * d) - s + d * atan(s / d);
}

double orc_seg_int_log(double xx, double xy, double ax, double ay, double bx, double by) {
  double lx = bx - ax, ly = by - ay, len = sqrt(lx * lx + ly * ly);
  double tx = lx / len, ty = ly / len, nx = ty, ny = -tx;
  double s1 = (ax - xx) * tx + (ay - xy) * ty, s2 = s1 + len;
  double d = (xx - ax) * nx + (xy - ay) * ny;
  return segF(s2, d) - segF(s1, d);
}

/* int over segment [a,b] of d/dn_y ln|x - y| ds_y with n the segment's outward normal
 * (tangent rotated clockwise).  d/dn_y ln|x-y| = -d/(s^2+d^2). */
double orc_seg_int_dlog(double xx, double xy, double ax, double ay, double bx, double by) {
  double lx = bx - ax, ly = by - ay, len = sqrt(lx * lx + ly * ly);
  double tx = lx / len, ty = ly / len, nx = ty, ny = -tx;
  double s1 = (ax - xx) * tx + (ay - xy) * ty, s2 = s1 + len;
  double d = (xx - ax) * nx + (xy - ay) * ny;
  if (d == 0.0) return 0.0;
  return -(atan(s2 / d) - atan(s1 / d));
}

/* Element e of 4n on the square [x0,x0+side]^2: endpoints (a, b) in traversal order. */
static void side_point(int sigma, double t, double x0, double y0, double side, double *x,
                       double *y) {
  switch (sigma) {
    case 0: *x = x0 + t; *y = y0; break;
    case 1: *x = x0 + side; *y = y0 + t; break;
    case 2: *x = x0 + side - t; *y = y0 + side; break;
    default: *x = x0; *y = y0 + side - t; break;
  }
}

void orc_elements(int n, double x0, double y0, double side, double *ax, double *ay, double *bx,
                  double *by, double *cx, double *cy) {
  const double el = side / n;
  for (int sg = 0; sg < 4; ++sg)
    for (int k = 0; k < n; ++k) {
      int e = sg * n + k;
      side_point(sg, k * el, x0, y0, side, &ax[e], &ay[e]);
      side_point(sg, (k + 1) * el, x0, y0, side, &bx[e], &by[e]);
      side_point(sg, (k + 0.5) * el, x0, y0, side, &cx[e], &cy[e]);
    }
}

/* Single-layer matrix S_mk = int_{Gamma_k} G(y_m, y) dGamma (left side of e:ubound)
 * and double-layer matrix K_mk = int_{Gamma_k} dG/dn(y_m, y) dGamma, both N_G x N_G,
 * row-major. */
void orc_bem_matrices(int n, double x0, double y0, double side, double *S, double *K) {
  const int NG = 4 * n;
  double *ax = malloc(sizeof(double) * NG * 6);
  double *ay = ax + NG, *bx = ay + NG, *by = bx + NG, *cx = by + NG, *cy = cx + NG;
  orc_elements(n, x0, y0, side, ax, ay, bx, by, cx, cy);
#pragma omp parallel for schedule(static)
  for (int m = 0; m < NG; ++m)
    for (int k = 0; k < NG; ++k) {
      if (S) S[(int64_t)m * NG + k] = -orc_seg_int_log(cx[m], cy[m], ax[k], ay[k], bx[k], by[k]) / (2.0 * PI_);
      if (K) K[(int64_t)m * NG + k] = -orc_seg_int_dlog(cx[m], cy[m], ax[k], ay[k], bx[k], by[k]) / (2.0 * PI_);
    }
  free(ax);
}

/* Selected rows of the two matrices of orc_bem_matrices: S[r][k] and K[r][k] for the
 * collocation indices rows[0..nr), each row N_G long (NULL skips a matrix).  Used to check
 * the boundary system S q = -(V r)|_Gamma of Eq. e:ubound at sampled collocation points of
 * grids whose full N_G x N_G matrices are too large to form. */
void orc_bem_rows(int n, double x0, double y0, double side, int nr, const int32_t *rows, double *S,
                  double *K) {
  const int NG = 4 * n;
  double *ax = malloc(sizeof(double) * NG * 6);
  double *ay = ax + NG, *bx = ay + NG, *by = bx + NG, *cx = by + NG, *cy = cx + NG;
  orc_elements(n, x0, y0, side, ax, ay, bx, by, cx, cy);
#pragma omp parallel for schedule(static)
  for (int t = 0; t < nr; ++t) {
    const int m = rows[t];
    for (int k = 0; k < NG; ++k) {
      if (S) S[(int64_t)t * NG + k] = -orc_seg_int_log(cx[m], cy[m], ax[k], ay[k], bx[k], by[k]) / (2.0 * PI_);
      if (K) K[(int64_t)t * NG + k] = -orc_seg_int_dlog(cx[m], cy[m], ax[k], ay[k], bx[k], by[k]) / (2.0 * PI_);
    }
  }
  free(ax);
}

/* Boundary-layer potentials of constant-element densities at targets off the boundary
 * (the two boundary integrals of Eq. e:uinter): sl[t] = sum_k q_k int_{Gamma_k} G(x_t, y)
 * dGamma_y and dl[t] = sum_k mu_k int_{Gamma_k} dG/dn_y(x_t, y) dGamma_y, with
 * G = -(1/2pi) ln|x - y|; q or mu NULL skips that sum. */
void orc_layers_at(int n, double x0, double y0, double side, const double *q, const double *mu, int nt,
                   const double *tx, const double *ty, double *sl, double *dl) {
  const int NG = 4 * n;
  double *ax = malloc(sizeof(double) * NG * 6);
  double *ay = ax + NG, *bx = ay + NG, *by = bx + NG, *cx = by + NG, *cy = cx + NG;
  orc_elements(n, x0, y0, side, ax, ay, bx, by, cx, cy);
#pragma omp parallel for schedule(static)
  for (int t = 0; t < nt; ++t) {
    double a = 0.0, b = 0.0;
    for (int k = 0; k < NG; ++k) {
      if (q) a += q[k] * orc_seg_int_log(tx[t], ty[t], ax[k], ay[k], bx[k], by[k]);
      if (mu) b += mu[k] * orc_seg_int_dlog(tx[t], ty[t], ax[k], ay[k], bx[k], by[k]);
    }
    if (sl) sl[t] = -a / (2.0 * PI_);
    if (dl) dl[t] = -b / (2.0 * PI_);
  }
  free(ax);
}

/* Dense LU with partial pivoting (Doolittle), in place; piv[i] = row swapped with i.
 * Returns 0, or 1 if a pivot is exactly zero. */
int orc_lu(int N, double *A, int32_t *piv) {
  for (int k = 0; k < N; ++k) {
    int pr = k;
    double best = fabs(A[(int64_t)k * N + k]);
    for (int i = k + 1; i < N; ++i)
      if (fabs(A[(int64_t)i * N + k]) > best) { best = fabs(A[(int64_t)i * N + k]); pr = i; }
    piv[k] = pr;
    if (best == 0.0) return 1;
    if (pr != k)
      for (int j = 0; j < N; ++j) {
        double t = A[(int64_t)k * N + j];
        A[(int64_t)k * N + j] = A[(int64_t)pr * N + j];
        A[(int64_t)pr * N + j] = t;
      }
    const double dk = A[(int64_t)k * N + k];
#pragma omp parallel for schedule(static)
    for (int i = k + 1; i < N; ++i) {
      double lik = A[(int64_t)i * N + k] / dk;
      A[(int64_t)i * N + k] = lik;
      for (int j = k + 1; j < N; ++j) A[(int64_t)i * N + j] -= lik * A[(int64_t)k * N + j];
    }
  }
  return 0;
}

void orc_lu_solve(int N, const double *LU, const int32_t *piv, double *x) {
  for (int k = 0; k < N; ++k)
    if (piv[k] != k) { double t = x[k]; x[k] = x[piv[k]]; x[piv[k]] = t; }
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < i; ++j) x[i] -= LU[(int64_t)i * N + j] * x[j];
  for (int i = N - 1; i >= 0; --i) {
    for (int j = i + 1; j < N; ++j) x[i] -= LU[(int64_t)i * N + j] * x[j];
    x[i] /= LU[(int64_t)i * N + i];
  }
}

/* Solves A^T x = b with the factors of orc_lu (P A = L U, so A^T = U^T L^T P): U^T y = b,
 * L^T w = y, then x = P^T w (the row swaps undone in reverse order). */
void orc_lu_solve_transpose(int N, const double *LU, const int32_t *piv, double *x) {
  for (int i = 0; i < N; ++i) {
    for (int j = 0; j < i; ++j) x[i] -= LU[(int64_t)j * N + i] * x[j];
    x[i] /= LU[(int64_t)i * N + i];
  }
  for (int i = N - 1; i >= 0; --i)
    for (int j = i + 1; j < N; ++j) x[i] -= LU[(int64_t)j * N + i] * x[j];
  for (int k = N - 1; k >= 0; --k)
    if (piv[k] != k) { double t = x[k]; x[k] = x[piv[k]]; x[piv[k]] = t; }
}

/* ======================================================================== */
/* 5. Tree (Sec. 5.1): split at centre lines until a cell holds at most      */
/*    leaf_max nodes.  On an n = m 2^L grid this gives the complete quadtree. */
/*    Bodies are ordered by Morton key (bits of i interleaved with bits of j, */
/*    i in the even positions).                                               */
/* ======================================================================== */

static uint32_t morton2(uint32_t ix, uint32_t iy) {
  uint32_t k = 0;
  for (int b = 0; b < 16; ++b) {
    k |= ((ix >> b) & 1u) << (2 * b);
    k |= ((iy >> b) & 1u) << (2 * b + 1);
  }
  return k;
}

static void demorton2(uint64_t k, int64_t *ix, int64_t *iy) {
  int64_t x = 0, y = 0;
  for (int b = 0; b < 31; ++b) {
    x |= (int64_t)((k >> (2 * b)) & 1u) << b;
    y |= (int64_t)((k >> (2 * b + 1)) & 1u) << b;
  }
  *ix = x;
  *iy = y;
}

void orc_morton_keys(int n, uint32_t *keys) {
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) keys[j * n + i] = morton2((uint32_t)i, (uint32_t)j);
}

static const uint32_t *g_sort_keys;
static int cmp_key_idx(const void *a, const void *b) {
  int32_t ia = *(const int32_t *)a, ib = *(const int32_t *)b;
  if (g_sort_keys[ia] != g_sort_keys[ib]) return g_sort_keys[ia] < g_sort_keys[ib] ? -1 : 1;
  return (ia > ib) - (ia < ib); /* ties keep input order: stable */
}

/* perm[k] = natural index of the k-th body in Morton order (stable). */
void orc_sort_perm(int N, const uint32_t *keys, int32_t *perm) {
  for (int k = 0; k < N; ++k) perm[k] = k;
  g_sort_keys = keys;
  qsort(perm, (size_t)N, sizeof(int32_t), cmp_key_idx);
}

/* Leaf level for leaf_max: the first level whose cells hold at most leaf_max nodes.
 * Returns -1 if a split would cut through a row of nodes (n not m 2^L). */
int orc_leaf_level(int n, int leaf_max) {
  int L = 0, s = n;
  while ((int64_t)s * s > leaf_max) {
    if (s % 2) return -1;
    s /= 2;
    ++L;
  }
  return L;
}

/* ======================================================================== */
/* 6. Dual tree traversal (Sec. 5.2), starting from (root, root):           */
/*    MAC(A,B) -> M2L(A <- B); else both leaves -> P2P(A <- B); else split.  */
/*    MAC: (R_A + R_B) < theta |c_A - c_B|, R = half-diagonal of the cell.   */
/*    Reading: with theta = a/b it is tested exactly in integers,             */
/*    2 b^2 (s_A + s_B)^2 < a^2 d^2 (half-widths s and centre distance d).    */
/*    Equal cells are both split (all 4x4 child pairs in Morton order).       */
/*    Boundary cells are runs of elements along one side (a binary tree per   */
/*    side, 2^l runs at level l); their R is the half-diagonal of the square  */
/*    circumscribing the run.                                                  */
/* ======================================================================== */

typedef struct {
  int32_t *v;
  int64_t n, cap;
  int w;
} vec_t;

static void vpush(vec_t *a, const int32_t *e) {
  if (a->n == a->cap) {
    a->cap = a->cap ? a->cap * 2 : 1024;
    a->v = realloc(a->v, sizeof(int32_t) * a->w * a->cap);
  }
  memcpy(a->v + a->n * a->w, e, sizeof(int32_t) * a->w);
  a->n++;
}

typedef struct {
  int n, m, L, p, tnum, tden, N, NG;
  double x0, y0, side, h;
  uint32_t *keys;
  int32_t *perm;
  int32_t *cell_start; /* all levels, cell (l,c) at (4^l-1)/3 + c */
  vec_t m2l, p2p, m2l_vb, p2p_vb;
  int64_t *m2l_first; /* CSR over targets of m2l (all levels) */
  int64_t *p2p_first; /* CSR over target leaves of p2p */
  int64_t *vb_first;  /* CSR over volume targets of m2l_vb */
  int64_t *pvb_first; /* CSR over volume leaves of p2p_vb */
  double *eax, *eay, *ebx, *eby, *ecx, *ecy;
  double *LU;
  int32_t *piv;
  int lu_ok;
  double *LUdl;      /* LU factors of -1/2 I + K (second-kind variant), made on first use */
  int32_t *pivdl;
  int dl_ok;
  /* operator of the Krylov solves: 0 five-point (Eq. e:axb), 1 five-point with the
   * variable coefficient acoef (Sec. 6.4), 2 Q1 stiffness (Sec. 6.1), whose residuals
   * the preconditioner takes through the inverse Q1 mass matrix (orc_q1_mass_solve) */
  int op;
  double *acoef;
} orc_prob;

static int64_t lev_off(int l) { return ((((int64_t)1) << (2 * l)) - 1) / 3; }
static int64_t blev_off(int l) { return 4 * ((((int64_t)1) << l) - 1); }

/* Volume cell geometry in units of h/2, relative to x0: centre (X,Y), half-width s. */
static void vcell(const orc_prob *P, int l, int64_t c, int64_t *X, int64_t *Y, int64_t *s) {
  int64_t a, b;
  demorton2((uint64_t)c, &a, &b);
  int64_t w = P->n >> l;
  *X = 2 * a * w + w + 1;
  *Y = 2 * b * w + w + 1;
  *s = w;
}

static int mac_vv(const orc_prob *P, int l, int64_t A, int64_t B) {
  int64_t XA, YA, sA, XB, YB, sB;
  vcell(P, l, A, &XA, &YA, &sA);
  vcell(P, l, B, &XB, &YB, &sB);
  __int128 d2 = (__int128)(XA - XB) * (XA - XB) + (__int128)(YA - YB) * (YA - YB);
  __int128 lhs = (__int128)2 * P->tden * P->tden * (sA + sB) * (sA + sB);
  return lhs < (__int128)P->tnum * P->tnum * d2;
}

static void dtt_vv(orc_prob *P, int l, int64_t A, int64_t B) {
  if (mac_vv(P, l, A, B)) {
    int32_t e[3] = {l, (int32_t)A, (int32_t)B};
    vpush(&P->m2l, e);
  } else if (l == P->L) {
    int32_t e[2] = {(int32_t)A, (int32_t)B};
    vpush(&P->p2p, e);
  } else {
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) dtt_vv(P, l + 1, 4 * A + i, 4 * B + j);
  }
}

/* Geometry in units u = h / 2^(L+1), origin (x0, y0). */
static void bcell_u(const orc_prob *P, int l, int sigma, int64_t k, int64_t *X, int64_t *Y,
                    int64_t *s) {
  int64_t np1 = P->n + 1, SL = np1 << (P->L + 1);
  int64_t t = (2 * k + 1) * np1 * (((int64_t)1) << (P->L - l));
  *s = np1 * (((int64_t)1) << (P->L - l));
  switch (sigma) {
    case 0: *X = t; *Y = 0; break;
    case 1: *X = SL; *Y = t; break;
    case 2: *X = SL - t; *Y = SL; break;
    default: *X = 0; *Y = SL - t; break;
  }
}

static int mac_vb(const orc_prob *P, int l, int64_t v, int sigma, int64_t k) {
  int64_t X, Y, s, BX, BY, bs;
  vcell(P, l, v, &X, &Y, &s);
  X <<= P->L; Y <<= P->L; s <<= P->L;
  bcell_u(P, l, sigma, k, &BX, &BY, &bs);
  __int128 d2 = (__int128)(X - BX) * (X - BX) + (__int128)(Y - BY) * (Y - BY);
  __int128 lhs = (__int128)2 * P->tden * P->tden * (__int128)(s + bs) * (s + bs);
  return lhs < (__int128)P->tnum * P->tnum * d2;
}

static void dtt_vb(orc_prob *P, int l, int64_t v, int sigma, int64_t k) {
  if (mac_vb(P, l, v, sigma, k)) {
    int32_t e[3] = {l, (int32_t)v, (int32_t)((int64_t)sigma * (((int64_t)1) << l) + k)};
    vpush(&P->m2l_vb, e);
  } else if (l == P->L) {
    int32_t e[2] = {(int32_t)v, (int32_t)((int64_t)sigma * (((int64_t)1) << l) + k)};
    vpush(&P->p2p_vb, e);
  } else {
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 2; ++j) dtt_vb(P, l + 1, 4 * v + i, sigma, 2 * k + j);
  }
}

static int cmp3(const void *a, const void *b) {
  const int32_t *x = a, *y = b;
  for (int i = 0; i < 3; ++i)
    if (x[i] != y[i]) return x[i] < y[i] ? -1 : 1;
  return 0;
}
static int cmp2(const void *a, const void *b) {
  const int32_t *x = a, *y = b;
  for (int i = 0; i < 2; ++i)
    if (x[i] != y[i]) return x[i] < y[i] ? -1 : 1;
  return 0;
}

/* CSR "first entry of each target" over a list whose column col holds targets sorted
 * ascending within each level block. key(t) = global index. */
static int64_t *csr_first(const vec_t *a, int64_t ntarget, int tcol, int lcol, int boundary) {
  int64_t *first = malloc(sizeof(int64_t) * (ntarget + 1));
  for (int64_t t = 0; t <= ntarget; ++t) first[t] = -1;
  int64_t *cnt = calloc((size_t)ntarget + 1, sizeof(int64_t));
  for (int64_t e = 0; e < a->n; ++e) {
    const int32_t *r = a->v + e * a->w;
    int64_t g = (lcol >= 0 ? (boundary ? blev_off(r[lcol]) : lev_off(r[lcol])) : 0) + r[tcol];
    cnt[g]++;
  }
  /* entries are grouped by (level, target) so a running offset works */
  int64_t off = 0;
  for (int64_t t = 0; t < ntarget; ++t) { first[t] = off; off += cnt[t]; }
  first[ntarget] = off;
  free(cnt);
  return first;
}

/* ======================================================================== */
/* Problem set-up (the analogue of PCSetUp, Sec. 7.1).                       */
/* ======================================================================== */

orc_prob *orc_create(int n, double x0, double y0, double side, int leaf_max, int p, int tnum,
                     int tden) {
  int L = orc_leaf_level(n, leaf_max);
  if (L < 0 || n < 2 || p < 1 || p > ORC_PMAX || tnum <= 0 || tden <= 0) return NULL;
  if ((n >> L) * (n >> L) > 1024) return NULL;
  binom_init();
  orc_prob *P = calloc(1, sizeof(orc_prob));
  P->n = n; P->L = L; P->m = n >> L; P->p = p; P->tnum = tnum; P->tden = tden;
  P->N = n * n; P->NG = 4 * n;
  P->x0 = x0; P->y0 = y0; P->side = side; P->h = side / (n + 1);
  P->keys = malloc(sizeof(uint32_t) * P->N);
  P->perm = malloc(sizeof(int32_t) * P->N);
  orc_morton_keys(n, P->keys);
  orc_sort_perm(P->N, P->keys, P->perm);
  /* cell ranges: a cell starts where the key prefix of its level first appears */
  int64_t ncell = lev_off(L + 1);
  P->cell_start = malloc(sizeof(int32_t) * ncell);
  for (int64_t c = 0; c < ncell; ++c) P->cell_start[c] = -1;
  int lg = 0;
  while ((1 << lg) < n) ++lg;
  for (int l = 0; l <= L; ++l) {
    int sh = 2 * (lg - l);
    for (int k = 0; k < P->N; ++k) {
      uint32_t c = P->keys[P->perm[k]] >> sh;
      if (k == 0 || c != (P->keys[P->perm[k - 1]] >> sh)) P->cell_start[lev_off(l) + c] = k;
    }
  }
  P->m2l.w = 3; P->p2p.w = 2; P->m2l_vb.w = 3; P->p2p_vb.w = 2;
  dtt_vv(P, 0, 0, 0);
  for (int sg = 0; sg < 4; ++sg) dtt_vb(P, 0, 0, sg, 0);
  qsort(P->m2l.v, (size_t)P->m2l.n, sizeof(int32_t) * 3, cmp3);
  qsort(P->p2p.v, (size_t)P->p2p.n, sizeof(int32_t) * 2, cmp2);
  qsort(P->m2l_vb.v, (size_t)P->m2l_vb.n, sizeof(int32_t) * 3, cmp3);
  qsort(P->p2p_vb.v, (size_t)P->p2p_vb.n, sizeof(int32_t) * 2, cmp2);
  P->m2l_first = csr_first(&P->m2l, ncell, 1, 0, 0);
  P->p2p_first = csr_first(&P->p2p, ((int64_t)1) << (2 * L), 0, -1, 0);
  P->vb_first = csr_first(&P->m2l_vb, ncell, 1, 0, 0);
  P->pvb_first = csr_first(&P->p2p_vb, ((int64_t)1) << (2 * L), 0, -1, 0);
  /* boundary elements, BEM matrix and its LU factors (Sec. 4.3) */
  int NG = P->NG;
  P->eax = malloc(sizeof(double) * NG * 6);
  P->eay = P->eax + NG; P->ebx = P->eay + NG; P->eby = P->ebx + NG;
  P->ecx = P->eby + NG; P->ecy = P->ecx + NG;
  orc_elements(n, x0, y0, side, P->eax, P->eay, P->ebx, P->eby, P->ecx, P->ecy);
  P->LU = malloc(sizeof(double) * (int64_t)NG * NG);
  P->piv = malloc(sizeof(int32_t) * NG);
  orc_bem_matrices(n, x0, y0, side, P->LU, NULL);
  P->lu_ok = (orc_lu(NG, P->LU, P->piv) == 0);
  P->op = 0;
  P->acoef = NULL;
  P->LUdl = NULL;
  P->pivdl = NULL;
  P->dl_ok = 0;
  return P;
}

void orc_destroy(orc_prob *P) {
  if (!P) return;
  free(P->keys); free(P->perm); free(P->cell_start);
  free(P->m2l.v); free(P->p2p.v); free(P->m2l_vb.v); free(P->p2p_vb.v);
  free(P->m2l_first); free(P->p2p_first); free(P->vb_first); free(P->pvb_first);
  free(P->eax); free(P->LU); free(P->piv); free(P->acoef); free(P->LUdl); free(P->pivdl);
  free(P);
}

/* Sizes: 0 L, 1 leaf side m, 2 #M2L, 3 #P2P, 4 #M2L vol-bnd, 5 #P2P vol-bnd, 6 N_Gamma,
 * 7 #cells, 8 LU ok. */
int64_t orc_query(const orc_prob *P, int what) {
  switch (what) {
    case 0: return P->L;
    case 1: return P->m;
    case 2: return P->m2l.n;
    case 3: return P->p2p.n;
    case 4: return P->m2l_vb.n;
    case 5: return P->p2p_vb.n;
    case 6: return P->NG;
    case 7: return lev_off(P->L + 1);
    case 8: return P->lu_ok;
    default: return -1;
  }
}

/* Copies: 0 keys (u32, natural order), 1 perm (i32), 2 cell_start (i32, all levels),
 * 3 m2l (i32 x3), 4 p2p (i32 x2), 5 m2l_vb (i32 x3), 6 p2p_vb (i32 x2). */
void orc_export(const orc_prob *P, int what, void *dst) {
  switch (what) {
    case 0: memcpy(dst, P->keys, sizeof(uint32_t) * P->N); break;
    case 1: memcpy(dst, P->perm, sizeof(int32_t) * P->N); break;
    case 2: memcpy(dst, P->cell_start, sizeof(int32_t) * lev_off(P->L + 1)); break;
    case 3: memcpy(dst, P->m2l.v, sizeof(int32_t) * 3 * P->m2l.n); break;
    case 4: memcpy(dst, P->p2p.v, sizeof(int32_t) * 2 * P->p2p.n); break;
    case 5: memcpy(dst, P->m2l_vb.v, sizeof(int32_t) * 3 * P->m2l_vb.n); break;
    case 6: memcpy(dst, P->p2p_vb.v, sizeof(int32_t) * 2 * P->p2p_vb.n); break;
    default: break;
  }
}

/* ---- geometry in physical units ---- */
static cplx vcentre(const orc_prob *P, int l, int64_t c) {
  int64_t X, Y, s;
  vcell(P, l, c, &X, &Y, &s);
  return (P->x0 + X * 0.5 * P->h) + I * (P->y0 + Y * 0.5 * P->h);
}
static cplx bcentre(const orc_prob *P, int l, int64_t sid) {
  int sg = (int)(sid >> l);
  int64_t k = sid & ((((int64_t)1) << l) - 1);
  double x, y, t = (k + 0.5) * P->side / (double)(((int64_t)1) << l);
  side_point(sg, t, P->x0, P->y0, P->side, &x, &y);
  return x + I * y;
}
static cplx node_z(const orc_prob *P, int idx) {
  return (P->x0 + (idx % P->n + 1) * P->h) + I * (P->y0 + (idx / P->n + 1) * P->h);
}

/* ======================================================================== */
/* 7. Preconditioner z = P^{-1} r (Sec. 3.2, Fig. f:flow_chart; Sec. 4.1).    */
/*    With u = 0 on Gamma, e:ubound reads  S q = -(V r)|_Gamma  and e:uinter    */
/*    reads  z = V r + int_Gamma q G dGamma  (q = dz/dn).                       */
/*    mode 0: every matrix-vector product done directly (Sec. 4.3).             */
/*    mode 1: every product done with the FMM of Sec. 5 (Sec. 4.3: "We also    */
/*    use the FMM to accelerate all other matrix-vector multiplications").      */
/*    Optional outputs (NULL to skip): vr = V r at the nodes, vr_col = V r at   */
/*    the collocation points, q, near = P2P part of V r, far = M2L part of V r. */
/* ======================================================================== */

static void apply_direct(orc_prob *P, const double *r, double *z, double *vr, double *vr_col,
                         double *qout) {
  const int n = P->n, N = P->N, NG = P->NG;
  const double h = P->h;
  double *Vr = malloc(sizeof(double) * N), *b = malloc(sizeof(double) * NG);
  orc_direct_V(n, P->x0, P->y0, P->side, r, Vr);
  orc_direct_V_at(n, P->x0, P->y0, P->side, r, NG, P->ecx, P->ecy, b);
  if (vr) memcpy(vr, Vr, sizeof(double) * N);
  if (vr_col) memcpy(vr_col, b, sizeof(double) * NG);
  for (int m = 0; m < NG; ++m) b[m] = -b[m];
  orc_lu_solve(NG, P->LU, P->piv, b); /* b <- q */
  if (qout) memcpy(qout, b, sizeof(double) * NG);
#pragma omp parallel for schedule(static)
  for (int i = 0; i < N; ++i) {
    double xi = P->x0 + (i % n + 1) * h, yi = P->y0 + (i / n + 1) * h, acc = 0.0;
    for (int k = 0; k < NG; ++k)
      acc += b[k] * orc_seg_int_log(xi, yi, P->eax[k], P->eay[k], P->ebx[k], P->eby[k]);
    z[i] = Vr[i] - acc / (2.0 * PI_);
  }
  free(Vr);
  free(b);
}

static void apply_fmm(orc_prob *P, const double *r, double *z, double *vr, double *vr_col,
                      double *qout, double *near_out, double *far_out) {
  const int p = P->p, L = P->L, N = P->N, NG = P->NG, n = P->n, m = P->m;
  const double h = P->h;
  const int64_t ncell = lev_off(L + 1), nleaf = ((int64_t)1) << (2 * L);
  const int64_t nb = blev_off(L + 1);
  cplx *M = calloc((size_t)(ncell * p), sizeof(cplx));
  cplx *Lv = calloc((size_t)(ncell * p), sizeof(cplx));
  cplx *Mb = calloc((size_t)(nb * p), sizeof(cplx));
  cplx *Lb = calloc((size_t)(nb * p), sizeof(cplx));
  double *w = malloc(sizeof(double) * N);
  double *phi_near = calloc(N, sizeof(double)), *phi_far = calloc(N, sizeof(double));
  double *phi_col = calloc(NG, sizeof(double)), *q = malloc(sizeof(double) * NG);
  double *phi_b = calloc(N, sizeof(double));
  for (int i = 0; i < N; ++i) w[i] = h * h * r[i]; /* quadrature weight of e:volume_integral */

  /* P2M at the leaves (Sec. 5.3 item 1) */
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < nleaf; ++c) {
    int s0 = P->cell_start[lev_off(L) + c];
    double px[1024], py[1024], f[1024];
    int np = m * m;
    for (int k = 0; k < np; ++k) {
      int idx = P->perm[s0 + k];
      cplx zz = node_z(P, idx);
      px[k] = creal(zz); py[k] = cimag(zz); f[k] = w[idx];
    }
    cplx zc = vcentre(P, L, c);
    orc_p2m(p, np, px, py, f, creal(zc), cimag(zc), M + (lev_off(L) + c) * p);
  }
  /* M2M upward (item 2) */
  for (int l = L - 1; l >= 0; --l) {
    int64_t nc = ((int64_t)1) << (2 * l);
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < nc; ++c) {
      cplx zM = vcentre(P, l, c);
      for (int ch = 0; ch < 4; ++ch) {
        int64_t cc = 4 * c + ch;
        m2m_(p, M + (lev_off(l + 1) + cc) * p, zM - vcentre(P, l + 1, cc), M + (lev_off(l) + c) * p);
      }
    }
  }
  /* (V r) at collocation points: M2L volume -> boundary, L2L along sides, L2P, P2P */
  for (int64_t e = 0; e < P->m2l_vb.n; ++e) {
    const int32_t *t = P->m2l_vb.v + 3 * e;
    int l = t[0];
    cplx zb = bcentre(P, l, t[2]);
    m2l_(p, M + (lev_off(l) + t[1]) * p, zb - vcentre(P, l, t[1]), Lb + (blev_off(l) + t[2]) * p);
  }
  for (int l = 0; l < L; ++l)
    for (int64_t sid = 0; sid < 4 * (((int64_t)1) << l); ++sid) {
      int sg = (int)(sid >> l);
      int64_t k = sid & ((((int64_t)1) << l) - 1);
      for (int ch = 0; ch < 2; ++ch) {
        int64_t cs = (int64_t)sg * (((int64_t)1) << (l + 1)) + 2 * k + ch;
        l2l_(p, Lb + (blev_off(l) + sid) * p, bcentre(P, l + 1, cs) - bcentre(P, l, sid),
                Lb + (blev_off(l + 1) + cs) * p);
      }
    }
  for (int64_t sid = 0; sid < 4 * (((int64_t)1) << L); ++sid) {
    int sg = (int)(sid >> L);
    int64_t k = sid & ((((int64_t)1) << L) - 1);
    cplx zb = bcentre(P, L, sid);
    for (int e = 0; e < m; ++e) {
      int g = sg * n + (int)k * m + e;
      phi_col[g] += l2p_(p, Lb + (blev_off(L) + sid) * p, (P->ecx[g] + I * P->ecy[g]) - zb);
    }
  }
  for (int64_t e = 0; e < P->p2p_vb.n; ++e) {
    const int32_t *t = P->p2p_vb.v + 2 * e;
    int sg = t[1] >> L, k = t[1] & ((1 << L) - 1);
    int s0 = P->cell_start[lev_off(L) + t[0]];
    for (int el = 0; el < m; ++el) {
      int g = sg * n + k * m + el;
      for (int j = 0; j < m * m; ++j) {
        int idx = P->perm[s0 + j];
        cplx d = (P->ecx[g] + I * P->ecy[g]) - node_z(P, idx);
        phi_col[g] += w[idx] * log(cabs(d));
      }
    }
  }
  /* BEM solve of e:ubound with u = 0 on Gamma */
  for (int g = 0; g < NG; ++g) q[g] = phi_col[g] / (2.0 * PI_); /* = -(V r)|_Gamma */
  if (vr_col)
    for (int g = 0; g < NG; ++g) vr_col[g] = -phi_col[g] / (2.0 * PI_);
  orc_lu_solve(NG, P->LU, P->piv, q);
  if (qout) memcpy(qout, q, sizeof(double) * NG);
  /* boundary multipoles: each element integrated exactly, int (zeta - c)^n ds */
  for (int64_t sid = 0; sid < 4 * (((int64_t)1) << L); ++sid) {
    int sg = (int)(sid >> L);
    int64_t k = sid & ((((int64_t)1) << L) - 1);
    cplx c = bcentre(P, L, sid), *Mo = Mb + (blev_off(L) + sid) * p;
    for (int el = 0; el < m; ++el) {
      int g = sg * n + (int)k * m + el;
      cplx za = (P->eax[g] + I * P->eay[g]) - c, zb = (P->ebx[g] + I * P->eby[g]) - c;
      cplx dz = zb - za;
      double len = cabs(dz);
      cplx e = dz / len;
      Mo[0] += q[g] * len;
      for (int kk = 1; kk < p; ++kk)
        Mo[kk] += -q[g] / kk * (ipow(zb, kk + 1) - ipow(za, kk + 1)) / ((kk + 1) * e);
    }
  }
  for (int l = L - 1; l >= 0; --l)
    for (int64_t sid = 0; sid < 4 * (((int64_t)1) << l); ++sid) {
      int sg = (int)(sid >> l);
      int64_t k = sid & ((((int64_t)1) << l) - 1);
      for (int ch = 0; ch < 2; ++ch) {
        int64_t cs = (int64_t)sg * (((int64_t)1) << (l + 1)) + 2 * k + ch;
        m2m_(p, Mb + (blev_off(l + 1) + cs) * p, bcentre(P, l, sid) - bcentre(P, l + 1, cs),
                Mb + (blev_off(l) + sid) * p);
      }
    }
  /* M2L into the volume locals (item 3): volume sources, then boundary sources */
  cplx *Lbv = calloc((size_t)(ncell * p), sizeof(cplx));
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t t = 0; t < ncell; ++t) {
    for (int64_t e = P->m2l_first[t]; e < P->m2l_first[t + 1]; ++e) {
      const int32_t *tr = P->m2l.v + 3 * e;
      int l = tr[0];
      m2l_(p, M + (lev_off(l) + tr[2]) * p, vcentre(P, l, tr[1]) - vcentre(P, l, tr[2]),
              Lv + (lev_off(l) + tr[1]) * p);
    }
    for (int64_t e = P->vb_first[t]; e < P->vb_first[t + 1]; ++e) {
      const int32_t *tr = P->m2l_vb.v + 3 * e;
      int l = tr[0];
      m2l_(p, Mb + (blev_off(l) + tr[2]) * p, vcentre(P, l, tr[1]) - bcentre(P, l, tr[2]),
              Lbv + (lev_off(l) + tr[1]) * p);
    }
  }
  /* L2L downward (item 4) */
  for (int l = 0; l < L; ++l) {
    int64_t nc = ((int64_t)1) << (2 * l);
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < nc; ++c)
      for (int ch = 0; ch < 4; ++ch) {
        int64_t cc = 4 * c + ch;
        cplx d = vcentre(P, l + 1, cc) - vcentre(P, l, c);
        l2l_(p, Lv + (lev_off(l) + c) * p, d, Lv + (lev_off(l + 1) + cc) * p);
        l2l_(p, Lbv + (lev_off(l) + c) * p, d, Lbv + (lev_off(l + 1) + cc) * p);
      }
  }
  /* L2P (item 5) and the near field: P2P between leaves, analytic element integrals */
#pragma omp parallel for schedule(dynamic, 8)
  for (int64_t c = 0; c < nleaf; ++c) {
    int s0 = P->cell_start[lev_off(L) + c];
    cplx zc = vcentre(P, L, c);
    for (int k = 0; k < m * m; ++k) {
      int i = P->perm[s0 + k];
      cplx zi = node_z(P, i);
      phi_far[i] = l2p_(p, Lv + (lev_off(L) + c) * p, zi - zc);
      double pb = l2p_(p, Lbv + (lev_off(L) + c) * p, zi - zc);
      double acc = 0.0;
      for (int64_t e = P->p2p_first[c]; e < P->p2p_first[c + 1]; ++e) {
        int sc = P->p2p.v[2 * e + 1];
        int t0 = P->cell_start[lev_off(L) + sc];
        for (int jj = 0; jj < m * m; ++jj) {
          int j = P->perm[t0 + jj];
          cplx zj = node_z(P, j);
          acc += w[j] * node_log(h, creal(zi), cimag(zi), creal(zj), cimag(zj), i == j);
        }
      }
      phi_near[i] = acc;
      for (int64_t e = P->pvb_first[c]; e < P->pvb_first[c + 1]; ++e) {
        int sid = P->p2p_vb.v[2 * e + 1];
        int sg = sid >> L, kk = sid & ((1 << L) - 1);
        for (int el = 0; el < m; ++el) {
          int g = sg * n + kk * m + el;
          pb += q[g] * orc_seg_int_log(creal(zi), cimag(zi), P->eax[g], P->eay[g], P->ebx[g], P->eby[g]);
        }
      }
      phi_b[i] = pb;
    }
  }
  for (int i = 0; i < N; ++i) {
    double vri = -(phi_near[i] + phi_far[i]) / (2.0 * PI_);
    if (vr) vr[i] = vri;
    if (near_out) near_out[i] = -phi_near[i] / (2.0 * PI_);
    if (far_out) far_out[i] = -phi_far[i] / (2.0 * PI_);
    z[i] = vri - phi_b[i] / (2.0 * PI_);
  }
  free(M); free(Lv); free(Mb); free(Lb); free(Lbv); free(w);
  free(phi_near); free(phi_far); free(phi_col); free(q); free(phi_b);
}

int orc_apply(orc_prob *P, int mode, const double *r, double *z, double *vr, double *vr_col,
              double *q, double *near_out, double *far_out) {
  if (!P->lu_ok) return 1;
  if (mode == 0) apply_direct(P, r, z, vr, vr_col, q);
  else apply_fmm(P, r, z, vr, vr_col, q, near_out, far_out);
  return 0;
}

/* ======================================================================== */
/* 7b. The boundary-integral solution with Dirichlet data g (Sec. 4.1):      */
/*     Eq. e:ubound  S q = (1/2 I + K) g - (V f)|_Gamma  for q = du/dn, then   */
/*     Eq. e:uinter  u = V f + int_Gamma q G - int_Gamma g dG/dn  in Omega,    */
/*     g and q constant on each element (values at the midpoints).  V f by    */
/*     the FMM (mode 1) or the direct sum (mode 0); the boundary integrals in  */
/*     closed form, summed directly.  out_q (optional) receives q.            */
/* ======================================================================== */

int orc_apply_bc(orc_prob *P, int mode, const double *f, const double *g, double *u, double *out_q) {
  if (!P->lu_ok) return 1;
  const int N = P->N, NG = P->NG, n = P->n;
  double *z = malloc(sizeof(double) * N), *vr = malloc(sizeof(double) * N);
  double *vc = malloc(sizeof(double) * NG), *q = malloc(sizeof(double) * NG);
  double *K = malloc(sizeof(double) * (int64_t)NG * NG);
  orc_apply(P, mode, f, z, vr, vc, NULL, NULL, NULL);
  orc_bem_matrices(n, P->x0, P->y0, P->side, NULL, K);
  for (int m = 0; m < NG; ++m) {
    double kg = 0.0;
    for (int k = 0; k < NG; ++k) kg += K[(int64_t)m * NG + k] * g[k];
    q[m] = 0.5 * g[m] + kg - vc[m];
  }
  orc_lu_solve(NG, P->LU, P->piv, q);
  if (out_q) memcpy(out_q, q, sizeof(double) * NG);
  const double h = P->h;
#pragma omp parallel for schedule(static)
  for (int i = 0; i < N; ++i) {
    const double xi = P->x0 + (i % n + 1) * h, yi = P->y0 + (i / n + 1) * h;
    double a = 0.0, b = 0.0;
    for (int k = 0; k < NG; ++k) {
      a += q[k] * orc_seg_int_log(xi, yi, P->eax[k], P->eay[k], P->ebx[k], P->eby[k]);
      b += g[k] * orc_seg_int_dlog(xi, yi, P->eax[k], P->eay[k], P->ebx[k], P->eby[k]);
    }
    u[i] = vr[i] - a / (2.0 * PI_) + b / (2.0 * PI_);
  }
  free(z); free(vr); free(vc); free(q); free(K);
  return 0;
}

/* ======================================================================== */
/* 7d. The transpose of the preconditioner, for gradients with respect to the */
/*     source weights.  P^{-1} r = V r + S_OG q with S q = -V_GO r (Eqs.       */
/*     e:ubound/e:uinter with z = 0 on Gamma), so                              */
/*     P^{-T} zb = V zb - V_GO^T S^{-T} S_OG^T zb: V is symmetric (G_ij = G_ji, */
/*     equal cell weights h^2); (S_OG^T zb)_k = sum_i zb_i int_k G(x_i, y);     */
/*     (V_GO^T c)_j = h^2 sum_m c_m G(y_m, x_j).  V zb by the FMM (mode 1) or   */
/*     the direct sum (mode 0); the boundary parts summed directly.            */
/* ======================================================================== */

int orc_apply_transpose(orc_prob *P, int mode, const double *zb, double *rb) {
  if (!P->lu_ok) return 1;
  const int N = P->N, NG = P->NG, n = P->n;
  const double h = P->h;
  double *z = malloc(sizeof(double) * N), *vr = malloc(sizeof(double) * N);
  double *t = calloc(NG, sizeof(double));
  orc_apply(P, mode, zb, z, vr, NULL, NULL, NULL, NULL);  /* vr = V zb */
#pragma omp parallel for schedule(static)
  for (int k = 0; k < NG; ++k) {
    double a = 0.0;
    for (int i = 0; i < N; ++i) {
      const double xi = P->x0 + (i % n + 1) * h, yi = P->y0 + (i / n + 1) * h;
      a += zb[i] * orc_seg_int_log(xi, yi, P->eax[k], P->eay[k], P->ebx[k], P->eby[k]);
    }
    t[k] = -a / (2.0 * PI_);
  }
  orc_lu_solve_transpose(NG, P->LU, P->piv, t);  /* t <- S^{-T} S_OG^T zb */
#pragma omp parallel for schedule(static)
  for (int j = 0; j < N; ++j) {
    const double xj = P->x0 + (j % n + 1) * h, yj = P->y0 + (j / n + 1) * h;
    double a = 0.0;
    for (int m = 0; m < NG; ++m) {
      const double dx = P->ecx[m] - xj, dy = P->ecy[m] - yj;
      a += t[m] * 0.5 * log(dx * dx + dy * dy);
    }
    rb[j] = vr[j] + h * h * a / (2.0 * PI_);  /* - V_GO^T t, G = -(1/2pi) ln r */
  }
  free(z); free(vr); free(t);
  return 0;
}

/* ======================================================================== */
/* 7c. Second-kind double-layer variant of the correction (a reading of the  */
/*     "double-layer boundary correction"): z = V r + w with w the double-     */
/*     layer potential of a density mu on Gamma, w(x) = int_Gamma mu dG/dn_y,  */
/*     whose limit from inside is (-1/2 I + K) mu; w = -(V r) on Gamma gives   */
/*     (-1/2 I + K) mu = -(V r)|_Gamma (a second-kind system), then w at the   */
/*     nodes by the closed-form element integrals.  out_mu (optional).         */
/* ======================================================================== */

int orc_apply_dl(orc_prob *P, int mode, const double *r, double *z, double *out_mu) {
  const int N = P->N, NG = P->NG, n = P->n;
  if (!P->LUdl) {
    P->LUdl = malloc(sizeof(double) * (int64_t)NG * NG);
    P->pivdl = malloc(sizeof(int32_t) * NG);
    orc_bem_matrices(n, P->x0, P->y0, P->side, NULL, P->LUdl);
    for (int m = 0; m < NG; ++m) P->LUdl[(int64_t)m * NG + m] -= 0.5;
    P->dl_ok = (orc_lu(NG, P->LUdl, P->pivdl) == 0);
  }
  if (!P->dl_ok || !P->lu_ok) return 1;
  double *zz = malloc(sizeof(double) * N), *vr = malloc(sizeof(double) * N);
  double *mu = malloc(sizeof(double) * NG);
  orc_apply(P, mode, r, zz, vr, mu, NULL, NULL, NULL); /* mu <- (V r)|_Gamma */
  for (int m = 0; m < NG; ++m) mu[m] = -mu[m];
  orc_lu_solve(NG, P->LUdl, P->pivdl, mu);
  if (out_mu) memcpy(out_mu, mu, sizeof(double) * NG);
  const double h = P->h;
#pragma omp parallel for schedule(static)
  for (int i = 0; i < N; ++i) {
    const double xi = P->x0 + (i % n + 1) * h, yi = P->y0 + (i / n + 1) * h;
    double b = 0.0;
    for (int k = 0; k < NG; ++k) b += mu[k] * orc_seg_int_dlog(xi, yi, P->eax[k], P->eay[k], P->ebx[k], P->eby[k]);
    z[i] = vr[i] - b / (2.0 * PI_);
  }
  free(zz); free(vr); free(mu);
  return 0;
}

/* ======================================================================== */
/* 8. Krylov methods (Sec. 3.1): CG, and GMRES(m) / FGMRES(m) with right    */
/*    preconditioning A P^{-1} y = b, x = P^{-1} y.  Zero initial iterate and  */
/*    a relative-residual stop (Sec. 6); the returned residual is the true     */
/*    ||b - A x|| / ||b|| recomputed at the end.                               */
/*    prec: 0 none, 1 direct form, 2 FMM form.  Iterations = P^{-1} actions    */
/*    inside the Krylov recurrence.                                            */
/* ======================================================================== */

static double dot(int N, const double *a, const double *b) {
  double s = 0.0;
  for (int i = 0; i < N; ++i) s += a[i] * b[i];
  return s;
}

/* Selects the operator of later solves (op 0, 1 with the (n+2)^2 coefficient a, or 2). */
int orc_set_operator(orc_prob *P, int op, const double *a) {
  if (op < 0 || op > 2 || (op == 1 && !a)) return 1;
  free(P->acoef);
  P->acoef = NULL;
  if (op == 1) {
    const size_t na = (size_t)(P->n + 2) * (P->n + 2);
    P->acoef = malloc(sizeof(double) * na);
    memcpy(P->acoef, a, sizeof(double) * na);
  }
  P->op = op;
  return 0;
}

static void op_apply(orc_prob *P, const double *x, double *y) {
  if (P->op == 1) orc_spmv5_var(P->n, P->h, P->acoef, x, y);
  else if (P->op == 2) orc_spmv_q1(P->n, x, y);
  else orc_spmv5(P->n, P->h, x, y);
}

/* prec: 0 none, 1 direct form, 2 FMM form, 3 FMM form with the second-kind double-layer
 * correction (orc_apply_dl) */
static void prec_apply(orc_prob *P, int prec, const double *r, double *z) {
  if (prec == 0) {
    memcpy(z, r, sizeof(double) * P->N);
    return;
  }
  double *c = NULL;
  if (P->op == 2) {  /* Q1: the preconditioner acts on the function M^{-1} r */
    c = malloc(sizeof(double) * P->N);
    orc_q1_mass_solve(P->n, P->h, r, c);
    r = c;
  }
  if (prec == 3) orc_apply_dl(P, 1, r, z, NULL);
  else orc_apply(P, prec == 1 ? 0 : 1, r, z, NULL, NULL, NULL, NULL, NULL);
  free(c);
}

static double true_relres(orc_prob *P, const double *b, const double *x, double bn) {
  double *t = malloc(sizeof(double) * P->N);
  op_apply(P, x, t);
  for (int i = 0; i < P->N; ++i) t[i] = b[i] - t[i];
  double r = sqrt(dot(P->N, t, t)) / bn;
  free(t);
  return r;
}

static int solve_cg(orc_prob *P, int prec, int maxit, double rtol, const double *b, double *x,
                    int *iters, double *hist) {
  const int N = P->N;
  double *r = malloc(sizeof(double) * N * 4), *zz = r + N, *pp = zz + N, *qq = pp + N;
  double bn = sqrt(dot(N, b, b));
  op_apply(P, x, r);
  for (int i = 0; i < N; ++i) r[i] = b[i] - r[i];
  int it = 0, conv = 0;
  if (hist) hist[0] = sqrt(dot(N, r, r)) / bn;
  if (sqrt(dot(N, r, r)) / bn <= rtol) conv = 1;
  prec_apply(P, prec, r, zz);
  memcpy(pp, zz, sizeof(double) * N);
  double rz = dot(N, r, zz);
  while (!conv && it < maxit) {
    op_apply(P, pp, qq);
    double alpha = rz / dot(N, pp, qq);
    for (int i = 0; i < N; ++i) { x[i] += alpha * pp[i]; r[i] -= alpha * qq[i]; }
    ++it;
    double rn = sqrt(dot(N, r, r)) / bn;
    if (hist) hist[it] = rn;
    if (rn <= rtol) { conv = 1; break; }
    prec_apply(P, prec, r, zz);
    double rz2 = dot(N, r, zz);
    double beta = rz2 / rz;
    rz = rz2;
    for (int i = 0; i < N; ++i) pp[i] = zz[i] + beta * pp[i];
  }
  *iters = it;
  free(r);
  return conv;
}

static int solve_gmres(orc_prob *P, int flexible, int prec, int restart, int maxit, double rtol,
                       const double *b, double *x, int *iters, double *hist) {
  const int N = P->N, m = restart;
  double *V = malloc(sizeof(double) * (int64_t)N * (m + 1));
  double *Z = malloc(sizeof(double) * (int64_t)N * (flexible ? m : 1));
  double *H = calloc((size_t)(m + 1) * m, sizeof(double));
  double *cs = malloc(sizeof(double) * m), *sn = malloc(sizeof(double) * m);
  double *g = malloc(sizeof(double) * (m + 1)), *y = malloc(sizeof(double) * m);
  double *w = malloc(sizeof(double) * N), *t = malloc(sizeof(double) * N);
  double bn = sqrt(dot(N, b, b));
  int it = 0, conv = 0;
  if (hist) hist[0] = 1.0;
  for (;;) {
    op_apply(P, x, w);
    for (int i = 0; i < N; ++i) w[i] = b[i] - w[i];
    double beta = sqrt(dot(N, w, w));
    if (beta / bn <= rtol) { conv = 1; break; }
    if (it >= maxit) break;
    for (int i = 0; i < N; ++i) V[i] = w[i] / beta;
    for (int i = 0; i <= m; ++i) g[i] = 0.0;
    g[0] = beta;
    int j = 0;
    for (; j < m && it < maxit; ++j) {
      double *zj = flexible ? Z + (int64_t)j * N : Z;
      prec_apply(P, prec, V + (int64_t)j * N, zj);
      op_apply(P, zj, w);
      for (int i = 0; i <= j; ++i) { /* modified Gram-Schmidt */
        double hij = dot(N, w, V + (int64_t)i * N);
        H[i * m + j] = hij;
        for (int k = 0; k < N; ++k) w[k] -= hij * V[(int64_t)i * N + k];
      }
      double hn = sqrt(dot(N, w, w));
      H[(j + 1) * m + j] = hn;
      if (hn > 0.0)
        for (int k = 0; k < N; ++k) V[(int64_t)(j + 1) * N + k] = w[k] / hn;
      for (int i = 0; i < j; ++i) { /* previous Givens rotations */
        double a = H[i * m + j], c = H[(i + 1) * m + j];
        H[i * m + j] = cs[i] * a + sn[i] * c;
        H[(i + 1) * m + j] = -sn[i] * a + cs[i] * c;
      }
      double a = H[j * m + j], c = H[(j + 1) * m + j], rr = hypot(a, c);
      cs[j] = a / rr; sn[j] = c / rr;
      H[j * m + j] = rr;
      H[(j + 1) * m + j] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      ++it;
      if (hist) hist[it] = fabs(g[j + 1]) / bn;
      if (fabs(g[j + 1]) / bn <= rtol || hn == 0.0) { ++j; break; }
    }
    for (int i = j - 1; i >= 0; --i) { /* back substitution H y = g */
      double s = g[i];
      for (int k = i + 1; k < j; ++k) s -= H[i * m + k] * y[k];
      y[i] = s / H[i * m + i];
    }
    if (flexible) {
      for (int i = 0; i < j; ++i)
        for (int k = 0; k < N; ++k) x[k] += y[i] * Z[(int64_t)i * N + k];
    } else {
      for (int k = 0; k < N; ++k) t[k] = 0.0;
      for (int i = 0; i < j; ++i)
        for (int k = 0; k < N; ++k) t[k] += y[i] * V[(int64_t)i * N + k];
      prec_apply(P, prec, t, w);
      for (int k = 0; k < N; ++k) x[k] += w[k];
    }
  }
  *iters = it;
  free(V); free(Z); free(H); free(cs); free(sn); free(g); free(y); free(w); free(t);
  return conv;
}

/* method: 0 CG, 1 GMRES(restart), 2 FGMRES(restart).  x holds the initial iterate.
 * Returns 1 if converged. */
int orc_solve(orc_prob *P, int method, int restart, int maxit, double rtol, int prec,
              const double *b, double *x, int *iters, double *relres, double *hist) {
  if (prec && !P->lu_ok) return -1;
  int conv;
  if (method == 0) conv = solve_cg(P, prec, maxit, rtol, b, x, iters, hist);
  else conv = solve_gmres(P, method == 2, prec, restart, maxit, rtol, b, x, iters, hist);
  *relres = true_relres(P, b, x, sqrt(dot(P->N, b, b)));
  return conv;
}
