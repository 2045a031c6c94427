/*
 * Red-black SOR oracle: plain, slow, single-threaded CPU code.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link
 * or call this file; only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark load it.  It shares no code, header or constant generator
 * with the CUDA path.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared (contraction off so that
 * every product and sum is rounded separately, in the order written here, on
 * both x86-64 and aarch64).
 *
 * Grid convention (paper, Section 3.1 and Section 3.4):
 *   interior side n, array side m = n+2, row-major U[i*m + j], i = row
 *   (row 0 is the "north" edge), j = column; the outer ring holds the
 *   Dirichlet data and is never written.  A cell is red when (i+j) is even
 *   and black when (i+j) is odd (Section 3.1, Figure 1).
 *   h = 1/(n+1); x_j = j*h, y_i = i*h.
 *
 * Update of one cell (Eq. 1 with the 5-point Gauss-Seidel value, Section 3.1):
 *   U <- (1-w)*U + (w/4)*( ((U_N + U_S) + (U_W + U_E)) + g ),   g = h^2 f,
 * for -Laplace(u) = f.  With f == NULL, g = 0 and the "+ g" term is omitted.
 *
 * Iteration (Algorithm 1): for iter = 1..max_iters: red phase over all red
 * interior cells, then black phase using the new red values.  When iter is a
 * multiple of K (check_every) the convergence quantity is tested:
 *   stop_mode 0: m = max over interior |U_iter - U_{iter-1}|   (Section 2.1)
 *   stop_mode 1: rho = max|r~| / max|b~| (scaled residual, see below)
 * and the loop stops with converged = 1 when it is strictly below tol.
 * Since every interior cell is updated exactly once per iteration, the
 * largest per-update change over the two phases equals the difference to the
 * snapshot Algorithm 1 copies before the red phase.
 *
 * Scaled residual (the stopping test of the precision workloads; the paper
 * itself stops on the change only):
 *   r~_ij = g_ij + (U_N + U_S + U_W + U_E) - 4 U_ij  over the interior,
 *   b~_ij = g_ij + (sum of the neighbours of (i,j) that lie on the ring),
 *   rho = max|r~| / max|b~|, or max|r~| when max|b~| == 0.
 * r~ equals h^2 (f - A u) with A the 5-point operator, so rho is the
 * infinity-norm relative residual with the boundary moved to the right side.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define IDX(i, j, m) ((size_t)(i) * (size_t)(m) + (size_t)(j))

/* g = h^2 f on the full (n+2)^2 array, zero on the ring; NULL f gives NULL. */
static double *make_g(int n, const double *f) {
  if (!f) return NULL;
  const int m = n + 2;
  const double h = 1.0 / (double)(n + 1);
  const double h2 = h * h;
  double *g = (double *)calloc((size_t)m * m, sizeof(double));
  if (!g) return NULL;
  for (int i = 1; i <= n; ++i)
    for (int j = 1; j <= n; ++j) g[IDX(i, j, m)] = h2 * f[(size_t)(i - 1) * n + (j - 1)];
  return g;
}

/* One colour phase in FP64 (Eq. 1); returns the largest |change|. */
static double phase_f64(int n, double *U, const double *g, double omega, int colour) {
  const int m = n + 2;
  const double a = 1.0 - omega, b = omega / 4.0;
  double dmax = 0.0;
  for (int i = 1; i <= n; ++i) {
    /* first interior column with (i+j) % 2 == colour */
    int j0 = ((i + 1) % 2 == colour) ? 1 : 2;
    for (int j = j0; j <= n; j += 2) {
      const double old = U[IDX(i, j, m)];
      double s = (U[IDX(i - 1, j, m)] + U[IDX(i + 1, j, m)]) + (U[IDX(i, j - 1, m)] + U[IDX(i, j + 1, m)]);
      if (g) s = s + g[IDX(i, j, m)];
      const double nu = a * old + b * s;
      U[IDX(i, j, m)] = nu;
      const double d = fabs(nu - old);
      if (d > dmax || d != d) dmax = d; /* a NaN, once seen, stays */
    }
  }
  return dmax;
}

/* Same phase in FP32 arithmetic (the reduced-precision sweep). */
static float phase_f32(int n, float *U, const float *g, float a, float b, int colour) {
  const int m = n + 2;
  float dmax = 0.0f;
  for (int i = 1; i <= n; ++i) {
    int j0 = ((i + 1) % 2 == colour) ? 1 : 2;
    for (int j = j0; j <= n; j += 2) {
      const float old = U[IDX(i, j, m)];
      float s = (U[IDX(i - 1, j, m)] + U[IDX(i + 1, j, m)]) + (U[IDX(i, j - 1, m)] + U[IDX(i, j + 1, m)]);
      if (g) s = s + g[IDX(i, j, m)];
      const float nu = a * old + b * s;
      U[IDX(i, j, m)] = nu;
      const float d = fabsf(nu - old);
      if (d > dmax || d != d) dmax = d;
    }
  }
  return dmax;
}

/* Scaled residual r~ (optionally stored in r, (n+2)^2, ring 0) and the two
 * infinity norms max|r~|, max|b~|. */
static void residual_f64(int n, const double *U, const double *g, double *r, double *rmax, double *bmax) {
  const int m = n + 2;
  double rm = 0.0, bm = 0.0;
  for (int i = 1; i <= n; ++i) {
    for (int j = 1; j <= n; ++j) {
      const double gij = g ? g[IDX(i, j, m)] : 0.0;
      const double nb = (U[IDX(i - 1, j, m)] + U[IDX(i + 1, j, m)]) + (U[IDX(i, j - 1, m)] + U[IDX(i, j + 1, m)]);
      const double res = (gij + nb) - 4.0 * U[IDX(i, j, m)];
      double bnd = 0.0;
      if (i == 1) bnd += U[IDX(0, j, m)];
      if (i == n) bnd += U[IDX(n + 1, j, m)];
      if (j == 1) bnd += U[IDX(i, 0, m)];
      if (j == n) bnd += U[IDX(i, n + 1, m)];
      const double bt = gij + bnd;
      if (r) r[IDX(i, j, m)] = res;
      const double ar = fabs(res), ab = fabs(bt);
      if (ar > rm || ar != ar) rm = ar;
      if (ab > bm) bm = ab;
    }
  }
  *rmax = rm;
  *bmax = bm;
}

static double rel(double rmax, double bmax) { return bmax > 0.0 ? rmax / bmax : rmax; }

/* Plain FP64 red-black SOR, Algorithm 1.
 *   u0: (n+2)^2 initial profile incl. ring; f: n*n interior source or NULL.
 *   u: (n+2)^2 output (may alias u0).  trace (optional, length max_iters)
 *   receives m_k for every iteration.  Returns 0, or -1 on bad arguments /
 *   allocation failure. */
int oracle_sor_f64(int n, double omega, const double *u0, const double *f, int max_iters, int check_every,
                   double tol, int stop_mode, int stall_window, double *u, int *iterations, int *converged,
                   double *final_maxdelta, double *final_resid_rel, double *trace) {
  if (n < 1 || max_iters < 0 || check_every < 1 || !u0 || !u) return -1;
  const int m = n + 2;
  if (u != u0) memcpy(u, u0, sizeof(double) * (size_t)m * m);
  double *g = make_g(n, f);
  if (f && !g) return -1;
  int it = 0, conv = 0;
  double mk = 0.0, rho = -1.0;
  /* stall rule (residual tests only): stop without convergence once
   * stall_window consecutive tests gave no new smallest rho while staying
   * within a factor 4 of it (a plateau at the attainable floor); a test
   * further above the smallest rho (the growth SOR shows early on) ends the
   * run of such tests */
  double best = HUGE_VAL;
  int run = 0;
  for (int k = 1; k <= max_iters; ++k) {
    const double dr = phase_f64(n, u, g, omega, 0); /* red   */
    const double db = phase_f64(n, u, g, omega, 1); /* black */
    mk = (dr > db || dr != dr) ? dr : db;
    if (trace) trace[k - 1] = mk;
    it = k;
    if (k % check_every == 0) {
      if (stop_mode == 0) {
        if (mk < tol) { conv = 1; break; }
      } else {
        double rm, bm;
        residual_f64(n, u, g, NULL, &rm, &bm);
        rho = rel(rm, bm);
        if (rho < tol) { conv = 1; break; }
        if (rho < best) { best = rho; run = 0; }
        else if (rho < 4.0 * best) { ++run; if (stall_window > 0 && run >= stall_window) break; }
        else run = 0;
      }
    }
  }
  {
    /* residual of the final iterate (equals the tested value on convergence) */
    double rm, bm;
    residual_f64(n, u, g, NULL, &rm, &bm);
    rho = rel(rm, bm);
  }
  free(g);
  if (iterations) *iterations = it;
  if (converged) *converged = conv;
  if (final_maxdelta) *final_maxdelta = mk;
  if (final_resid_rel) *final_resid_rel = rho;
  return 0;
}

/* Plain red-black SOR carried out in FP32 arithmetic and storage (the
 * reduced-precision sweep).  Coefficients are rounded once to FP32:
 * a = (float)(1 - w), b = (float)(w / 4); the source is rounded once,
 * gf = (float)(h^2 f).  u0 / u are FP64 arrays (converted on entry / exit).
 * Stops on max|change| only (stop_mode 0 semantics). */
int oracle_sor_f32(int n, double omega, const double *u0, const double *f, int max_iters, int check_every,
                   double tol, double *u, int *iterations, int *converged, double *final_maxdelta, double *trace) {
  if (n < 1 || max_iters < 0 || check_every < 1 || !u0 || !u) return -1;
  const int m = n + 2;
  const size_t cells = (size_t)m * m;
  float *U = (float *)malloc(sizeof(float) * cells);
  float *G = NULL;
  if (!U) return -1;
  for (size_t c = 0; c < cells; ++c) U[c] = (float)u0[c];
  double *g = make_g(n, f);
  if (g) {
    G = (float *)malloc(sizeof(float) * cells);
    if (!G) { free(U); free(g); return -1; }
    for (size_t c = 0; c < cells; ++c) G[c] = (float)g[c];
    free(g);
  }
  const float a = (float)(1.0 - omega), b = (float)(omega / 4.0);
  int it = 0, conv = 0;
  float mk = 0.0f;
  for (int k = 1; k <= max_iters; ++k) {
    const float dr = phase_f32(n, U, G, a, b, 0);
    const float db = phase_f32(n, U, G, a, b, 1);
    mk = (dr > db || dr != dr) ? dr : db;
    if (trace) trace[k - 1] = (double)mk;
    it = k;
    if (k % check_every == 0 && (double)mk < tol) { conv = 1; break; }
  }
  for (size_t c = 0; c < cells; ++c) u[c] = (double)U[c];
  free(U);
  free(G);
  if (iterations) *iterations = it;
  if (converged) *converged = conv;
  if (final_maxdelta) *final_maxdelta = (double)mk;
  return 0;
}

/* Scaled residual of u (FP64) with optional r output ((n+2)^2, ring 0). */
int oracle_residual(int n, const double *u, const double *f, double *r, double *rmax, double *bmax) {
  if (n < 1 || !u || !rmax || !bmax) return -1;
  double *g = make_g(n, f);
  if (f && !g) return -1;
  residual_f64(n, u, g, r, rmax, bmax);
  free(g);
  return 0;
}

/* Defect correction with reduced-precision inner sweeps.
 *   u <- u0; loop over outer steps:
 *     r~ = g + sum_nb(u) - 4u (FP64), rho = max|r~|/max|b~|; stop if rho < tol
 *       or when outer == max_outer;
 *     d  <- 0 on the whole (n+2)^2 array (its ring stays 0);
 *     inner_sweeps red-black SOR iterations on A d = r~ with rhs
 *       (float)r~ (already scaled by h^2) in FP32 (inner_f32 != 0) or FP64;
 *     u_interior += (double)d.
 * In exact arithmetic one outer step equals inner_sweeps plain SOR
 * iterations on u (same splitting, error map M^s).  Outputs: outer steps
 * done, total inner sweeps, final rho.  trace (optional, length max_outer+1)
 * receives rho per residual evaluation. */
int oracle_refine(int n, double omega, const double *u0, const double *f, int inner_sweeps, int inner_f32,
                  double tol, int max_outer, int stall_window, double *u, int *outer_steps, int *sweeps,
                  int *converged, double *final_resid_rel, double *trace) {
  if (n < 1 || inner_sweeps < 1 || max_outer < 0 || !u0 || !u) return -1;
  const int m = n + 2;
  const size_t cells = (size_t)m * m;
  if (u != u0) memcpy(u, u0, sizeof(double) * cells);
  double *g = make_g(n, f);
  double *r = (double *)calloc(cells, sizeof(double));
  double *d64 = (double *)calloc(cells, sizeof(double));
  float *d32 = (float *)calloc(cells, sizeof(float));
  float *r32 = (float *)calloc(cells, sizeof(float));
  if ((f && !g) || !r || !d64 || !d32 || !r32) {
    free(g); free(r); free(d64); free(d32); free(r32);
    return -1;
  }
  const float a32 = (float)(1.0 - omega), b32 = (float)(omega / 4.0);
  int outer = 0, conv = 0;
  double rho = 0.0, best = HUGE_VAL;
  int run = 0;
  for (;;) {
    double rm, bm;
    residual_f64(n, u, g, r, &rm, &bm);
    rho = rel(rm, bm);
    if (trace) trace[outer] = rho;
    if (rho < tol) { conv = 1; break; }
    if (outer == max_outer) break;
    /* stall rule, as in oracle_sor_f64 */
    if (rho < best) { best = rho; run = 0; }
    else if (rho < 4.0 * best) { ++run; if (stall_window > 0 && run >= stall_window) break; }
    else run = 0;
    if (inner_f32) {
      for (size_t c = 0; c < cells; ++c) { d32[c] = 0.0f; r32[c] = (float)r[c]; }
      for (int s = 0; s < inner_sweeps; ++s) {
        (void)phase_f32(n, d32, r32, a32, b32, 0);
        (void)phase_f32(n, d32, r32, a32, b32, 1);
      }
      for (int i = 1; i <= n; ++i)
        for (int j = 1; j <= n; ++j) u[IDX(i, j, m)] = u[IDX(i, j, m)] + (double)d32[IDX(i, j, m)];
    } else {
      memset(d64, 0, sizeof(double) * cells);
      for (int s = 0; s < inner_sweeps; ++s) {
        (void)phase_f64(n, d64, r, omega, 0);
        (void)phase_f64(n, d64, r, omega, 1);
      }
      for (int i = 1; i <= n; ++i)
        for (int j = 1; j <= n; ++j) u[IDX(i, j, m)] = u[IDX(i, j, m)] + d64[IDX(i, j, m)];
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

/* ---------------------------------------------------------------------------
 * Block two-colour SOR (block-parallel SOR).
 *
 * Section 3.1 names block-parallel SOR beside red-black and multi-colour SOR
 * as a parallel form of SOR, citing other work, and does not define it; the
 * reading taken here:
 *   - the interior is tiled into blocks of by rows x bx columns: block
 *     (I, J) holds rows 1 + I*by .. min(n, (I+1)*by) and columns
 *     1 + J*bx .. min(n, (J+1)*bx) (the last blocks of a row or column are
 *     clipped at n);
 *   - block (I, J) has colour (I + J) mod 2, so blocks of one colour touch
 *     only at corners and the 5-point stencil couples a block only to itself
 *     and to blocks of the other colour;
 *   - one iteration updates every colour-0 block, then every colour-1 block;
 *     inside a block the cells are updated one at a time in row-major order
 *     with the update of Eq. 1 (the expression and rounding order of
 *     phase_f64), each reading the newest value of every neighbour.
 * The blocks of a colour are independent, so they may run in any order or
 * at once (the parallelism of the method); they are taken here in row-major
 * block order.  by = bx = 1 gives red-black SOR (colour (i + j) mod 2, red
 * first); one block covering the interior gives SOR in natural row-major
 * order.  Each interior cell is updated once per iteration, so the largest
 * per-update change is again the difference between successive iterates.
 * ------------------------------------------------------------------------- */
static double block_phase_f64(int n, double *U, const double *g, double omega, int by, int bx, int colour) {
  const int m = n + 2;
  const double a = 1.0 - omega, b = omega / 4.0;
  const int nbr = (n + by - 1) / by, nbc = (n + bx - 1) / bx;
  double dmax = 0.0;
  for (int I = 0; I < nbr; ++I) {
    for (int J = 0; J < nbc; ++J) {
      if ((I + J) % 2 != colour) continue;
      const int ilast = (I + 1) * by < n ? (I + 1) * by : n;
      const int jlast = (J + 1) * bx < n ? (J + 1) * bx : n;
      for (int i = 1 + I * by; i <= ilast; ++i) {
        for (int j = 1 + J * bx; j <= jlast; ++j) {
          const double old = U[IDX(i, j, m)];
          double s = (U[IDX(i - 1, j, m)] + U[IDX(i + 1, j, m)]) + (U[IDX(i, j - 1, m)] + U[IDX(i, j + 1, m)]);
          if (g) s = s + g[IDX(i, j, m)];
          const double nu = a * old + b * s;
          U[IDX(i, j, m)] = nu;
          const double d = fabs(nu - old);
          if (d > dmax || d != d) dmax = d;
        }
      }
    }
  }
  return dmax;
}

/* Block two-colour SOR in FP64 with the loop and stopping test of
 * oracle_sor_f64 (test every K iterations, strict <; stop_mode 0 on the
 * largest change, 1 on the scaled residual; no stall rule).  by, bx >= 1.
 * Returns 0, or -1 on bad arguments / allocation failure. */
int oracle_sor_block_f64(int n, int by, int bx, double omega, const double *u0, const double *f, int max_iters,
                         int check_every, double tol, int stop_mode, double *u, int *iterations, int *converged,
                         double *final_maxdelta, double *final_resid_rel, double *trace) {
  if (n < 1 || by < 1 || bx < 1 || max_iters < 0 || check_every < 1 || !u0 || !u) return -1;
  const int m = n + 2;
  if (u != u0) memcpy(u, u0, sizeof(double) * (size_t)m * m);
  double *g = make_g(n, f);
  if (f && !g) return -1;
  int it = 0, conv = 0;
  double mk = 0.0, rho = -1.0;
  for (int k = 1; k <= max_iters; ++k) {
    const double d0 = block_phase_f64(n, u, g, omega, by, bx, 0);
    const double d1 = block_phase_f64(n, u, g, omega, by, bx, 1);
    mk = (d0 > d1 || d0 != d0) ? d0 : d1;
    if (trace) trace[k - 1] = mk;
    it = k;
    if (k % check_every == 0) {
      if (stop_mode == 0) {
        if (mk < tol) { conv = 1; break; }
      } else {
        double rm, bm;
        residual_f64(n, u, g, NULL, &rm, &bm);
        rho = rel(rm, bm);
        if (rho < tol) { conv = 1; break; }
      }
    }
  }
  {
    double rm, bm;
    residual_f64(n, u, g, NULL, &rm, &bm);
    rho = rel(rm, bm);
  }
  free(g);
  if (iterations) *iterations = it;
  if (converged) *converged = conv;
  if (final_maxdelta) *final_maxdelta = mk;
  if (final_resid_rel) *final_resid_rel = rho;
  return 0;
}

/* One colour phase of block two-colour SOR in FP32 arithmetic (the block
 * order of block_phase_f64, the expression and rounding of phase_f32). */
static float block_phase_f32(int n, float *U, const float *g, float a, float b, int by, int bx, int colour) {
  const int m = n + 2;
  const int nbr = (n + by - 1) / by, nbc = (n + bx - 1) / bx;
  float dmax = 0.0f;
  for (int I = 0; I < nbr; ++I) {
    for (int J = 0; J < nbc; ++J) {
      if ((I + J) % 2 != colour) continue;
      const int ilast = (I + 1) * by < n ? (I + 1) * by : n;
      const int jlast = (J + 1) * bx < n ? (J + 1) * bx : n;
      for (int i = 1 + I * by; i <= ilast; ++i) {
        for (int j = 1 + J * bx; j <= jlast; ++j) {
          const float old = U[IDX(i, j, m)];
          float s = (U[IDX(i - 1, j, m)] + U[IDX(i + 1, j, m)]) + (U[IDX(i, j - 1, m)] + U[IDX(i, j + 1, m)]);
          if (g) s = s + g[IDX(i, j, m)];
          const float nu = a * old + b * s;
          U[IDX(i, j, m)] = nu;
          const float d = fabsf(nu - old);
          if (d > dmax || d != d) dmax = d;
        }
      }
    }
  }
  return dmax;
}

/* Block two-colour SOR in FP32 arithmetic and storage, with the conventions
 * of oracle_sor_f32 (u0 rounded to FP32 on entry, coefficients (float)(1-w)
 * and (float)(w/4), the source rounded once as (float)(h^2 f), stop on
 * max|change| only, the result widened to FP64 on exit). */
int oracle_sor_block_f32(int n, int by, int bx, double omega, const double *u0, const double *f, int max_iters,
                         int check_every, double tol, double *u, int *iterations, int *converged,
                         double *final_maxdelta, double *trace) {
  if (n < 1 || by < 1 || bx < 1 || max_iters < 0 || check_every < 1 || !u0 || !u) return -1;
  const int m = n + 2;
  const size_t cells = (size_t)m * m;
  float *U = (float *)malloc(sizeof(float) * cells);
  float *G = NULL;
  if (!U) return -1;
  for (size_t c = 0; c < cells; ++c) U[c] = (float)u0[c];
  double *g = make_g(n, f);
  if (f && !g) { free(U); return -1; }
  if (g) {
    G = (float *)malloc(sizeof(float) * cells);
    if (!G) { free(U); free(g); return -1; }
    for (size_t c = 0; c < cells; ++c) G[c] = (float)g[c];
    free(g);
  }
  const float a = (float)(1.0 - omega), b = (float)(omega / 4.0);
  int it = 0, conv = 0;
  float mk = 0.0f;
  for (int k = 1; k <= max_iters; ++k) {
    const float d0 = block_phase_f32(n, U, G, a, b, by, bx, 0);
    const float d1 = block_phase_f32(n, U, G, a, b, by, bx, 1);
    mk = (d0 > d1 || d0 != d0) ? d0 : d1;
    if (trace) trace[k - 1] = (double)mk;
    it = k;
    if (k % check_every == 0 && (double)mk < tol) { conv = 1; break; }
  }
  for (size_t c = 0; c < cells; ++c) u[c] = (double)U[c];
  free(U);
  free(G);
  if (iterations) *iterations = it;
  if (converged) *converged = conv;
  if (final_maxdelta) *final_maxdelta = (double)mk;
  return 0;
}
