/*
 * Red-black SOR oracle on 3D grids: plain, slow, single-threaded CPU code.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link
 * or call this file; only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark load it.  It shares no code, header or constant generator
 * with the CUDA path.
 *
 * The paper solves the 2D problem and names the 3D grid as its next step
 * (Section 5, Conclusion and Future Work).  This file carries the same method
 * to a cube: Algorithm 1 with the cell update of Eq. 1, the Gauss-Seidel value
 * now taken from the 7-point stencil.
 *
 * Grid convention: interior side n, array side m = n+2, U[(k*m + i)*m + j],
 * k = plane (z), i = row (y), j = column (x); the outer shell holds the
 * Dirichlet data and is never written.  A cell is red when (i+j+k) is even
 * and black otherwise; the red phase runs first.  h = 1/(n+1).
 *
 * Update of one cell (Eq. 1, 7-point Gauss-Seidel value), -Laplace(u) = f:
 *   U <- (1-w)*U + (w/6)*( (((U_N + U_S) + (U_W + U_E)) + (U_D + U_U)) + g ),
 * with N/S = rows i-1/i+1, W/E = columns j-1/j+1, D/U = planes k-1/k+1 and
 * g = h^2 f (the "+ g" term is omitted when f == NULL).  The summation order
 * is part of the definition: the GPU's exact-order path follows it.
 *
 * Convergence (Algorithm 1, Section 2.1): on iterations that are multiples of
 * K, stop_mode 0 tests m = max |U_k - U_{k-1}| (the largest per-update
 * change, each cell being updated once per iteration) and stop_mode 1 the
 * scaled residual rho = max|r~| / max|b~| with
 *   r~ = g + (sum of the six neighbours) - 6 U,
 *   b~ = g + (sum of the neighbours that lie on the shell),
 * rho = max|r~| when max|b~| == 0; strict comparison with tol.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define IDX3(k, i, j, m) (((size_t)(k) * (size_t)(m) + (size_t)(i)) * (size_t)(m) + (size_t)(j))

/* g = h^2 f on the full (n+2)^3 array, zero on the shell; NULL f gives NULL. */
static double *make_g3(int n, const double *f) {
  if (!f) return NULL;
  const int m = n + 2;
  const double h = 1.0 / (double)(n + 1);
  const double h2 = h * h;
  double *g = (double *)calloc((size_t)m * m * m, sizeof(double));
  if (!g) return NULL;
  for (int k = 1; k <= n; ++k)
    for (int i = 1; i <= n; ++i)
      for (int j = 1; j <= n; ++j)
        g[IDX3(k, i, j, m)] = h2 * f[((size_t)(k - 1) * n + (i - 1)) * n + (j - 1)];
  return g;
}

/* One colour phase in FP64; returns the largest |change|. */
static double phase3_f64(int n, double *U, const double *g, double omega, int colour) {
  const int m = n + 2;
  const double a = 1.0 - omega, b = omega / 6.0;
  double dmax = 0.0;
  for (int k = 1; k <= n; ++k) {
    for (int i = 1; i <= n; ++i) {
      /* first interior column with (i+j+k) % 2 == colour */
      const int j0 = ((i + k + 1) % 2 == colour) ? 1 : 2;
      for (int j = j0; j <= n; j += 2) {
        const size_t c = IDX3(k, i, j, m);
        const double old = U[c];
        double s = ((U[IDX3(k, i - 1, j, m)] + U[IDX3(k, i + 1, j, m)]) + (U[c - 1] + U[c + 1])) +
                   (U[IDX3(k - 1, i, j, m)] + U[IDX3(k + 1, i, j, m)]);
        if (g) s = s + g[c];
        const double nu = a * old + b * s;
        U[c] = nu;
        const double d = fabs(nu - old);
        if (d > dmax || d != d) dmax = d; /* a NaN, once seen, stays */
      }
    }
  }
  return dmax;
}

/* Same phase in FP32 arithmetic and storage. */
static float phase3_f32(int n, float *U, const float *g, float a, float b, int colour) {
  const int m = n + 2;
  float dmax = 0.0f;
  for (int k = 1; k <= n; ++k) {
    for (int i = 1; i <= n; ++i) {
      const int j0 = ((i + k + 1) % 2 == colour) ? 1 : 2;
      for (int j = j0; j <= n; j += 2) {
        const size_t c = IDX3(k, i, j, m);
        const float old = U[c];
        float s = ((U[IDX3(k, i - 1, j, m)] + U[IDX3(k, i + 1, j, m)]) + (U[c - 1] + U[c + 1])) +
                  (U[IDX3(k - 1, i, j, m)] + U[IDX3(k + 1, i, j, m)]);
        if (g) s = s + g[c];
        const float nu = a * old + b * s;
        U[c] = nu;
        const float d = fabsf(nu - old);
        if (d > dmax || d != d) dmax = d;
      }
    }
  }
  return dmax;
}

/* Scaled residual r~ (optionally stored in r, (n+2)^3, shell 0) and the
 * infinity norms max|r~|, max|b~|. */
static void residual3_f64(int n, const double *U, const double *g, double *r, double *rmax, double *bmax) {
  const int m = n + 2;
  double rm = 0.0, bm = 0.0;
  for (int k = 1; k <= n; ++k) {
    for (int i = 1; i <= n; ++i) {
      for (int j = 1; j <= n; ++j) {
        const size_t c = IDX3(k, i, j, m);
        const double gc = g ? g[c] : 0.0;
        const double nb = ((U[IDX3(k, i - 1, j, m)] + U[IDX3(k, i + 1, j, m)]) + (U[c - 1] + U[c + 1])) +
                          (U[IDX3(k - 1, i, j, m)] + U[IDX3(k + 1, i, j, m)]);
        const double res = (gc + nb) - 6.0 * U[c];
        double bnd = 0.0;
        if (i == 1) bnd += U[IDX3(k, 0, j, m)];
        if (i == n) bnd += U[IDX3(k, n + 1, j, m)];
        if (j == 1) bnd += U[IDX3(k, i, 0, m)];
        if (j == n) bnd += U[IDX3(k, i, n + 1, m)];
        if (k == 1) bnd += U[IDX3(0, i, j, m)];
        if (k == n) bnd += U[IDX3(n + 1, i, j, m)];
        const double bt = gc + bnd;
        if (r) r[c] = res;
        const double ar = fabs(res), ab = fabs(bt);
        if (ar > rm || ar != ar) rm = ar;
        if (ab > bm) bm = ab;
      }
    }
  }
  *rmax = rm;
  *bmax = bm;
}

static double rel3(double rmax, double bmax) { return bmax > 0.0 ? rmax / bmax : rmax; }

/* Plain FP64 red-black SOR on the cube (Algorithm 1).
 *   u0: (n+2)^3 initial values incl. the shell; f: n^3 interior source or
 *   NULL.  u: (n+2)^3 output (may alias u0).  trace (optional, length
 *   max_iters) receives m_k for every iteration.  Returns 0, or -1 on bad
 *   arguments / allocation failure. */
int oracle_sor3d_f64(int n, double omega, const double *u0, const double *f, int max_iters, int check_every,
                     double tol, int stop_mode, int stall_window, double *u, int *iterations, int *converged, double *final_maxdelta,
                     double *final_resid_rel, double *trace) {
  if (n < 1 || max_iters < 0 || check_every < 1 || stall_window < 0 || !u0 || !u) return -1;
  const int m = n + 2;
  const size_t cells = (size_t)m * m * m;
  if (u != u0) memcpy(u, u0, sizeof(double) * cells);
  double *g = make_g3(n, f);
  if (f && !g) return -1;
  int it = 0, conv = 0, run = 0;
  double mk = 0.0, rho = -1.0, best = HUGE_VAL;
  for (int k = 1; k <= max_iters; ++k) {
    const double dr = phase3_f64(n, u, g, omega, 0); /* red   */
    const double db = phase3_f64(n, u, g, omega, 1); /* black */
    mk = (dr > db || dr != dr) ? dr : db;
    if (trace) trace[k - 1] = mk;
    it = k;
    if (k % check_every == 0) {
      if (stop_mode == 0) {
        if (mk < tol) { conv = 1; break; }
      } else {
        double rm, bm;
        residual3_f64(n, u, g, NULL, &rm, &bm);
        rho = rel3(rm, bm);
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
    residual3_f64(n, u, g, NULL, &rm, &bm);
    rho = rel3(rm, bm);
  }
  free(g);
  if (iterations) *iterations = it;
  if (converged) *converged = conv;
  if (final_maxdelta) *final_maxdelta = mk;
  if (final_resid_rel) *final_resid_rel = rho;
  return 0;
}

/* The same iteration in FP32 arithmetic and storage: a = (float)(1 - w),
 * b = (float)(w / 6), gf = (float)(h^2 f), each rounded once.  u0 / u are
 * FP64 arrays (converted on entry / exit).  Stops on max|change| only. */
int oracle_sor3d_f32(int n, double omega, const double *u0, const double *f, int max_iters, int check_every,
                     double tol, double *u, int *iterations, int *converged, double *final_maxdelta, double *trace) {
  if (n < 1 || max_iters < 0 || check_every < 1 || !u0 || !u) return -1;
  const int m = n + 2;
  const size_t cells = (size_t)m * m * m;
  float *U = (float *)malloc(sizeof(float) * cells);
  float *G = NULL;
  if (!U) return -1;
  for (size_t c = 0; c < cells; ++c) U[c] = (float)u0[c];
  double *g = make_g3(n, f);
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
  const float a = (float)(1.0 - omega), b = (float)(omega / 6.0);
  int it = 0, conv = 0;
  float mk = 0.0f;
  for (int k = 1; k <= max_iters; ++k) {
    const float dr = phase3_f32(n, U, G, a, b, 0);
    const float db = phase3_f32(n, U, G, a, b, 1);
    mk = (dr > db || dr != dr) ? dr : db;
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

/* Scaled residual of a cube (see the header): r (optional, (n+2)^3) and the
 * two infinity norms.  Returns 0 or -1. */
int oracle_residual3d(int n, const double *u, const double *f, double *r, double *rmax, double *bmax) {
  if (n < 1 || !u || !rmax || !bmax) return -1;
  double *g = make_g3(n, f);
  if (f && !g) return -1;
  if (r) memset(r, 0, sizeof(double) * (size_t)(n + 2) * (n + 2) * (n + 2));
  residual3_f64(n, u, g, r, rmax, bmax);
  free(g);
  return 0;
}

/* Defect correction on a cube (the 2D oracle_refine carried to the 7-point
 * stencil):
 *   u <- u0; loop over outer steps:
 *     r~ = g + sum_nb(u) - 6u (FP64), rho = max|r~|/max|b~|; stop if
 *       rho < tol or when outer == max_outer;
 *     d  <- 0 on the whole (n+2)^3 array (its shell stays 0);
 *     inner_sweeps red-black SOR iterations on A d = r~ with right side
 *       (float)r~ (already scaled by h^2) in FP32 (inner_f32 != 0) or r~ in
 *       FP64, a = (float)(1 - w), b = (float)(w / 6) in FP32;
 *     u_interior += (double)d.
 * In exact arithmetic one outer step equals inner_sweeps plain SOR
 * iterations on u (same splitting, error map M^s).  Outputs: outer steps
 * done, total inner sweeps, final rho; trace (optional, length max_outer+1)
 * receives rho per residual evaluation. */
int oracle_refine3d(int n, double omega, const double *u0, const double *f, int inner_sweeps, int inner_f32,
                    double tol, int max_outer, int stall_window, double *u, int *outer_steps, int *sweeps, int *converged,
                    double *final_resid_rel, double *trace) {
  if (n < 1 || inner_sweeps < 1 || max_outer < 0 || stall_window < 0 || !u0 || !u) return -1;
  const int m = n + 2;
  const size_t cells = (size_t)m * m * m;
  if (u != u0) memcpy(u, u0, sizeof(double) * cells);
  double *g = make_g3(n, f);
  double *r = (double *)calloc(cells, sizeof(double));
  double *d64 = (double *)calloc(cells, sizeof(double));
  float *d32 = (float *)calloc(cells, sizeof(float));
  float *r32 = (float *)calloc(cells, sizeof(float));
  if ((f && !g) || !r || !d64 || !d32 || !r32) {
    free(g); free(r); free(d64); free(d32); free(r32);
    return -1;
  }
  const float a32 = (float)(1.0 - omega), b32 = (float)(omega / 6.0);
  int outer = 0, conv = 0, run = 0;
  double rho = 0.0, best = HUGE_VAL;
  for (;;) {
    double rm, bm;
    residual3_f64(n, u, g, r, &rm, &bm);
    rho = rel3(rm, bm);
    if (trace) trace[outer] = rho;
    if (rho < tol) { conv = 1; break; }
    if (outer == max_outer) break;
    /* the stall rule, as in the plain solve */
    if (rho < best) { best = rho; run = 0; }
    else if (rho < 4.0 * best) { ++run; if (stall_window > 0 && run >= stall_window) break; }
    else run = 0;
    if (inner_f32) {
      for (size_t c = 0; c < cells; ++c) { d32[c] = 0.0f; r32[c] = (float)r[c]; }
      for (int s = 0; s < inner_sweeps; ++s) {
        (void)phase3_f32(n, d32, r32, a32, b32, 0);
        (void)phase3_f32(n, d32, r32, a32, b32, 1);
      }
      for (int k = 1; k <= n; ++k)
        for (int i = 1; i <= n; ++i)
          for (int j = 1; j <= n; ++j) u[IDX3(k, i, j, m)] = u[IDX3(k, i, j, m)] + (double)d32[IDX3(k, i, j, m)];
    } else {
      memset(d64, 0, sizeof(double) * cells);
      for (int s = 0; s < inner_sweeps; ++s) {
        (void)phase3_f64(n, d64, r, omega, 0);
        (void)phase3_f64(n, d64, r, omega, 1);
      }
      for (int k = 1; k <= n; ++k)
        for (int i = 1; i <= n; ++i)
          for (int j = 1; j <= n; ++j) u[IDX3(k, i, j, m)] = u[IDX3(k, i, j, m)] + d64[IDX3(k, i, j, m)];
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
