/*
 * Four-colour SOR on the 9-point stencil: plain, slow, single-threaded CPU
 * code.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link
 * or call this file; only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark load it.  It shares no code, header or constant generator
 * with the CUDA path.
 *
 * Section 3.1 names multi-colour SOR next to red-black SOR as a parallel
 * ordering.  Two colours suffice for the 5-point stencil; the compact 9-point
 * stencil also couples diagonal neighbours, and four colours are needed so
 * that no cell has a neighbour of its own colour:
 *   colour c = 2 (i & 1) + (j & 1)   (0: even row, even column; 1: even, odd;
 *                                     2: odd, even; 3: odd, odd),
 * updated in the order 0, 1, 2, 3 within one iteration.
 *
 * Grid as in the 2D oracle: interior side n, array side m = n+2, row-major
 * U[i*m + j], the ring holds the Dirichlet data, h = 1/(n+1).
 *
 * Operator: the compact 9-point Laplacian
 *   (4 (U_N + U_S + U_W + U_E) + (U_NW + U_NE + U_SW + U_SE) - 20 U) / (6 h^2),
 * exact on harmonic polynomials up to degree 5.  For -Laplace(u) = f the cell
 * equation is 20 U = 4 s4 + sd + g with g = 6 h^2 f, and the SOR update
 * (Eq. 1 with this Gauss-Seidel value) is, summed in this order,
 *   s4 = (U_N + U_S) + (U_W + U_E),   sd = (U_NW + U_NE) + (U_SW + U_SE),
 *   s  = (4 s4 + sd) [+ g],           U <- (1-w) U + (w/20) s.
 *
 * Convergence (Algorithm 1, Section 2.1): on iterations that are multiples of
 * K, stop_mode 0 tests max |change| over the four phases, stop_mode 1 the
 * scaled residual rho = max|r~| / max|b~| with
 *   r~ = (g + (4 s4 + sd)) - 20 U,
 *   b~ = g + (4 bnd4 + bndd),  bnd4 / bndd = the ring neighbours among the
 *        edge (N, S, W, E) / diagonal (NW, NE, SW, SE) ones, summed in that
 *        order,
 * rho = max|r~| when max|b~| == 0; strict comparison with tol.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define AT(U, i, j, m) (U)[(size_t)(i) * (size_t)(m) + (size_t)(j)]

/* g = 6 h^2 f on the full (n+2)^2 array, zero on the ring. */
static double *make_g9(int n, const double *f) {
  if (!f) return NULL;
  const int m = n + 2;
  const double h = 1.0 / (double)(n + 1);
  const double s = 6.0 * (h * h);
  double *g = (double *)calloc((size_t)m * m, sizeof(double));
  if (!g) return NULL;
  for (int i = 1; i <= n; ++i)
    for (int j = 1; j <= n; ++j) AT(g, i, j, m) = s * f[(size_t)(i - 1) * n + (j - 1)];
  return g;
}

/* One colour phase in FP64; returns the largest |change|. */
static double phase9_f64(int n, double *U, const double *g, double omega, int colour) {
  const int m = n + 2;
  const double a = 1.0 - omega, b = omega / 20.0;
  const int pi = colour >> 1, pj = colour & 1;
  double dmax = 0.0;
  for (int i = 1; i <= n; ++i) {
    if ((i & 1) != pi) continue;
    for (int j = 1; j <= n; ++j) {
      if ((j & 1) != pj) continue;
      const double old = AT(U, i, j, m);
      const double s4 = (AT(U, i - 1, j, m) + AT(U, i + 1, j, m)) + (AT(U, i, j - 1, m) + AT(U, i, j + 1, m));
      const double sd =
          (AT(U, i - 1, j - 1, m) + AT(U, i - 1, j + 1, m)) + (AT(U, i + 1, j - 1, m) + AT(U, i + 1, j + 1, m));
      double s = 4.0 * s4 + sd;
      if (g) s = s + AT(g, i, j, m);
      const double nu = a * old + b * s;
      AT(U, i, j, m) = nu;
      const double d = fabs(nu - old);
      if (d > dmax || d != d) dmax = d;
    }
  }
  return dmax;
}

static float phase9_f32(int n, float *U, const float *g, float a, float b, int colour) {
  const int m = n + 2;
  const int pi = colour >> 1, pj = colour & 1;
  float dmax = 0.0f;
  for (int i = 1; i <= n; ++i) {
    if ((i & 1) != pi) continue;
    for (int j = 1; j <= n; ++j) {
      if ((j & 1) != pj) continue;
      const float old = AT(U, i, j, m);
      const float s4 = (AT(U, i - 1, j, m) + AT(U, i + 1, j, m)) + (AT(U, i, j - 1, m) + AT(U, i, j + 1, m));
      const float sd =
          (AT(U, i - 1, j - 1, m) + AT(U, i - 1, j + 1, m)) + (AT(U, i + 1, j - 1, m) + AT(U, i + 1, j + 1, m));
      float s = 4.0f * s4 + sd;
      if (g) s = s + AT(g, i, j, m);
      const float nu = a * old + b * s;
      AT(U, i, j, m) = nu;
      const float d = fabsf(nu - old);
      if (d > dmax || d != d) dmax = d;
    }
  }
  return dmax;
}

static void residual9_f64(int n, const double *U, const double *g, double *r, double *rmax, double *bmax) {
  const int m = n + 2;
  double rm = 0.0, bm = 0.0;
  for (int i = 1; i <= n; ++i) {
    for (int j = 1; j <= n; ++j) {
      const double gc = g ? AT(g, i, j, m) : 0.0;
      const double s4 = (AT(U, i - 1, j, m) + AT(U, i + 1, j, m)) + (AT(U, i, j - 1, m) + AT(U, i, j + 1, m));
      const double sd =
          (AT(U, i - 1, j - 1, m) + AT(U, i - 1, j + 1, m)) + (AT(U, i + 1, j - 1, m) + AT(U, i + 1, j + 1, m));
      const double res = (gc + (4.0 * s4 + sd)) - 20.0 * AT(U, i, j, m);
      double b4 = 0.0, bd = 0.0;
      if (i == 1) b4 += AT(U, 0, j, m);
      if (i == n) b4 += AT(U, n + 1, j, m);
      if (j == 1) b4 += AT(U, i, 0, m);
      if (j == n) b4 += AT(U, i, n + 1, m);
      if (i == 1 || j == 1) bd += AT(U, i - 1, j - 1, m);
      if (i == 1 || j == n) bd += AT(U, i - 1, j + 1, m);
      if (i == n || j == 1) bd += AT(U, i + 1, j - 1, m);
      if (i == n || j == n) bd += AT(U, i + 1, j + 1, m);
      const double bt = gc + (4.0 * b4 + bd);
      if (r) AT(r, i, j, m) = res;
      const double ar = fabs(res), ab = fabs(bt);
      if (ar > rm || ar != ar) rm = ar;
      if (ab > bm) bm = ab;
    }
  }
  *rmax = rm;
  *bmax = bm;
}

static double rel9(double rmax, double bmax) { return bmax > 0.0 ? rmax / bmax : rmax; }

/* FP64 four-colour SOR (Algorithm 1 with four phases per iteration).
 * Arguments as oracle_sor_f64 (without the stall rule). */
int oracle_sor9_f64(int n, double omega, const double *u0, const double *f, int max_iters, int check_every,
                    double tol, int stop_mode, int stall_window, double *u, int *iterations, int *converged,
                    double *final_maxdelta, double *final_resid_rel, double *trace) {
  if (n < 1 || max_iters < 0 || check_every < 1 || stall_window < 0 || !u0 || !u) return -1;
  const int m = n + 2;
  if (u != u0) memcpy(u, u0, sizeof(double) * (size_t)m * m);
  double *g = make_g9(n, f);
  if (f && !g) return -1;
  int it = 0, conv = 0, run = 0;
  double mk = 0.0, rho = -1.0, best = HUGE_VAL;
  for (int k = 1; k <= max_iters; ++k) {
    mk = 0.0;
    for (int c = 0; c < 4; ++c) {
      const double d = phase9_f64(n, u, g, omega, c);
      if (d > mk || d != d) mk = d;
    }
    if (trace) trace[k - 1] = mk;
    it = k;
    if (k % check_every == 0) {
      if (stop_mode == 0) {
        if (mk < tol) { conv = 1; break; }
      } else {
        double rm, bm;
        residual9_f64(n, u, g, NULL, &rm, &bm);
        rho = rel9(rm, bm);
        if (rho < tol) { conv = 1; break; }
        /* the stall rule of the 2D oracle: a plateau at the attainable
         * floor, stall_window tests without a new smallest rho within a
         * factor 4 of it, ends the run unconverged */
        if (rho < best) { best = rho; run = 0; }
        else if (rho < 4.0 * best) { ++run; if (stall_window > 0 && run >= stall_window) break; }
        else run = 0;
      }
    }
  }
  {
    double rm, bm;
    residual9_f64(n, u, g, NULL, &rm, &bm);
    rho = rel9(rm, bm);
  }
  free(g);
  if (iterations) *iterations = it;
  if (converged) *converged = conv;
  if (final_maxdelta) *final_maxdelta = mk;
  if (final_resid_rel) *final_resid_rel = rho;
  return 0;
}

/* The same iteration in FP32: a = (float)(1 - w), b = (float)(w / 20),
 * gf = (float)(6 h^2 f), each rounded once; u0 / u in FP64. */
int oracle_sor9_f32(int n, double omega, const double *u0, const double *f, int max_iters, int check_every,
                    double tol, double *u, int *iterations, int *converged, double *final_maxdelta, double *trace) {
  if (n < 1 || max_iters < 0 || check_every < 1 || !u0 || !u) return -1;
  const int m = n + 2;
  const size_t cells = (size_t)m * m;
  float *U = (float *)malloc(sizeof(float) * cells);
  float *G = NULL;
  if (!U) return -1;
  for (size_t c = 0; c < cells; ++c) U[c] = (float)u0[c];
  double *g = make_g9(n, f);
  if (f && !g) {
    free(U);
    return -1;
  }
  if (g) {
    G = (float *)malloc(sizeof(float) * cells);
    if (!G) {
      free(U);
      free(g);
      return -1;
    }
    for (size_t c = 0; c < cells; ++c) G[c] = (float)g[c];
  }
  const float a = (float)(1.0 - omega), b = (float)(omega / 20.0);
  int it = 0, conv = 0;
  float mk = 0.0f;
  for (int k = 1; k <= max_iters; ++k) {
    mk = 0.0f;
    for (int c = 0; c < 4; ++c) {
      const float d = phase9_f32(n, U, G, a, b, c);
      if (d > mk || d != d) mk = d;
    }
    if (trace) trace[k - 1] = (double)mk;
    it = k;
    if (k % check_every == 0 && (double)mk < tol) {
      conv = 1;
      break;
    }
  }
  for (size_t c = 0; c < cells; ++c) u[c] = (double)U[c];
  free(U);
  free(G);
  free(g);
  if (iterations) *iterations = it;
  if (converged) *converged = conv;
  if (final_maxdelta) *final_maxdelta = (double)mk;
  return 0;
}

int oracle_residual9(int n, const double *u, const double *f, double *r, double *rmax, double *bmax) {
  if (n < 1 || !u || !rmax || !bmax) return -1;
  double *g = make_g9(n, f);
  if (f && !g) return -1;
  if (r) memset(r, 0, sizeof(double) * (size_t)(n + 2) * (n + 2));
  residual9_f64(n, u, g, r, rmax, bmax);
  free(g);
  return 0;
}

/* Defect correction with the four-colour 9-point sweeps (the 2D
 * oracle_refine carried to this stencil):
 *   u <- u0; loop over outer steps:
 *     r~ = (g + (4 s4 + sd)) - 20u (FP64), rho = max|r~|/max|b~|; stop if
 *       rho < tol or when outer == max_outer;
 *     d  <- 0 on the whole (n+2)^2 array (its ring stays 0);
 *     inner_sweeps four-colour iterations on A d = r~ with right side
 *       (float)r~ in FP32 (inner_f32 != 0, a = (float)(1 - w),
 *       b = (float)(w / 20)) or r~ in FP64;
 *     u_interior += (double)d.
 * In exact arithmetic one outer step equals inner_sweeps plain iterations on
 * u.  Outputs: outer steps done, total inner sweeps, final rho; trace
 * (optional, length max_outer+1) receives rho per residual evaluation. */
int oracle_refine9(int n, double omega, const double *u0, const double *f, int inner_sweeps, int inner_f32,
                   double tol, int max_outer, int stall_window, double *u, int *outer_steps, int *sweeps, int *converged,
                   double *final_resid_rel, double *trace) {
  if (n < 1 || inner_sweeps < 1 || max_outer < 0 || stall_window < 0 || !u0 || !u) return -1;
  const int m = n + 2;
  const size_t cells = (size_t)m * m;
  if (u != u0) memcpy(u, u0, sizeof(double) * cells);
  double *g = make_g9(n, f);
  double *r = (double *)calloc(cells, sizeof(double));
  double *d64 = (double *)calloc(cells, sizeof(double));
  float *d32 = (float *)calloc(cells, sizeof(float));
  float *r32 = (float *)calloc(cells, sizeof(float));
  if ((f && !g) || !r || !d64 || !d32 || !r32) {
    free(g); free(r); free(d64); free(d32); free(r32);
    return -1;
  }
  const float a32 = (float)(1.0 - omega), b32 = (float)(omega / 20.0);
  int outer = 0, conv = 0, run = 0;
  double rho = 0.0, best = HUGE_VAL;
  for (;;) {
    double rm, bm;
    residual9_f64(n, u, g, r, &rm, &bm);
    rho = rel9(rm, bm);
    if (trace) trace[outer] = rho;
    if (rho < tol) { conv = 1; break; }
    if (outer == max_outer) break;
    /* the stall rule, as in the plain solve */
    if (rho < best) { best = rho; run = 0; }
    else if (rho < 4.0 * best) { ++run; if (stall_window > 0 && run >= stall_window) break; }
    else run = 0;
    if (inner_f32) {
      for (size_t c = 0; c < cells; ++c) { d32[c] = 0.0f; r32[c] = (float)r[c]; }
      for (int s = 0; s < inner_sweeps; ++s)
        for (int colour = 0; colour < 4; ++colour) (void)phase9_f32(n, d32, r32, a32, b32, colour);
      for (int i = 1; i <= n; ++i)
        for (int j = 1; j <= n; ++j) AT(u, i, j, m) = AT(u, i, j, m) + (double)AT(d32, i, j, m);
    } else {
      memset(d64, 0, sizeof(double) * cells);
      for (int s = 0; s < inner_sweeps; ++s)
        for (int colour = 0; colour < 4; ++colour) (void)phase9_f64(n, d64, r, omega, colour);
      for (int i = 1; i <= n; ++i)
        for (int j = 1; j <= n; ++j) AT(u, i, j, m) = AT(u, i, j, m) + AT(d64, i, j, m);
    }
    ++outer;
  }
  free(g); free(r); free(d64); free(d32); free(r32);
  if (outer_steps) *outer_steps = outer;
  if (sweeps) *sweeps = outer * inner_sweeps;
  if (converged) *converged = conv;
  if (final_resid_rel) *final_resid_rel = rho;
  return 0;
}
