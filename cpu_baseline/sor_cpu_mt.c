/*
 * Multithreaded CPU red-black SOR: the all-core CPU baseline of the
 * benchmark.  It is a measurement tool, not part of the solver library and
 * not the oracle (the oracle stays single-threaded and plain).
 *
 * The paper parallelises red-black SOR over P worker threads: within one
 * colour phase every update reads only the other colour, so the rows of a
 * phase are split among the threads, and a barrier separates the red phase
 * from the black one (Section 3.1, Section 3.2; Table 1 times P = 1..8).
 * This file does the same with POSIX threads: thread t owns a contiguous band
 * of interior rows, runs the red phase on its band, waits at a barrier, runs
 * the black phase, waits again; the largest |change| of the iteration is the
 * maximum of the per-thread maxima (Section 2.1), tested every K iterations
 * (Section 3.3).
 *
 * Every cell update is evaluated as
 *   U <- (1-w)*U + (w/4)*( ((U_N + U_S) + (U_W + U_E)) + g ),   g = h^2 f,
 * with each product and sum rounded on its own (built with contraction off),
 * and the updates of one colour are independent, so the result does not
 * depend on the number of threads: it equals the single-threaded iteration
 * bit for bit.  Layout: natural row-major (n+2)^2 array, row 0 north, ring =
 * Dirichlet data (never written); red cells have (i+j) even.
 */
#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#define AT(U, i, j, m) ((U)[(size_t)(i) * (size_t)(m) + (size_t)(j)])

typedef struct {
  int n, max_iters, check_every, nthreads;
  double omega, tol;
  double *u;        /* (n+2)^2 iterate */
  const double *g;  /* (n+2)^2 h^2 f (ring 0) or NULL */
  pthread_barrier_t bar;
  pthread_mutex_t mu;  /* start gate: workers wait until every thread exists */
  pthread_cond_t cv;
  int gate;            /* 0: wait, 1: run, -1: give up (a thread could not be created) */
  double *tmax;     /* per-thread max |change| of the current iteration */
  int stop;         /* set by thread 0 between iterations */
  int iters, conv;
  double mk;
} shared_t;

typedef struct {
  shared_t *s;
  int t, i0, i1; /* interior rows [i0, i1) */
} worker_t;

/* One colour phase over rows [i0, i1); returns the largest |change|
 * (a NaN, once seen, is kept). */
static double phase_rows(shared_t *s, int i0, int i1, int colour) {
  const int n = s->n, m = n + 2;
  const double a = 1.0 - s->omega, b = s->omega / 4.0;
  double *U = s->u;
  const double *g = s->g;
  double dmax = 0.0;
  for (int i = i0; i < i1; ++i) {
    const int j0 = ((i + 1) % 2 == colour) ? 1 : 2;
    for (int j = j0; j <= n; j += 2) {
      const double old = AT(U, i, j, m);
      double sum = (AT(U, i - 1, j, m) + AT(U, i + 1, j, m)) + (AT(U, i, j - 1, m) + AT(U, i, j + 1, m));
      if (g) sum = sum + AT(g, i, j, m);
      const double nu = a * old + b * sum;
      AT(U, i, j, m) = nu;
      const double d = fabs(nu - old);
      if (d > dmax || d != d) dmax = d;
    }
  }
  return dmax;
}

static void *worker(void *arg) {
  worker_t *w = (worker_t *)arg;
  shared_t *s = w->s;
  pthread_mutex_lock(&s->mu);
  while (s->gate == 0) pthread_cond_wait(&s->cv, &s->mu);
  const int gate = s->gate;
  pthread_mutex_unlock(&s->mu);
  if (gate < 0) return NULL;
  for (int k = 1; k <= s->max_iters; ++k) {
    const double dr = phase_rows(s, w->i0, w->i1, 0);
    pthread_barrier_wait(&s->bar);
    const double db = phase_rows(s, w->i0, w->i1, 1);
    s->tmax[w->t] = (dr > db || dr != dr) ? dr : db;
    pthread_barrier_wait(&s->bar);
    if (w->t == 0) {
      double mk = s->tmax[0];
      for (int t = 1; t < s->nthreads; ++t)
        if (s->tmax[t] > mk || s->tmax[t] != s->tmax[t]) mk = s->tmax[t];
      s->mk = mk;
      s->iters = k;
      if (k % s->check_every == 0 && mk < s->tol) {
        s->conv = 1;
        s->stop = 1;
      }
    }
    pthread_barrier_wait(&s->bar);
    if (s->stop) break;
  }
  return NULL;
}

/* Red-black SOR with the max|change| stop, on `threads` threads.
 *   u0: (n+2)^2 initial profile incl. ring; f: n*n interior source or NULL;
 *   u: (n+2)^2 output (may alias u0).  Returns 0, or -1 on bad arguments,
 *   allocation or thread failure. */
int cpu_sor_f64_mt(int n, double omega, const double *u0, const double *f, int max_iters, int check_every,
                   double tol, int threads, double *u, int *iterations, int *converged, double *final_maxdelta) {
  if (n < 1 || max_iters < 0 || check_every < 1 || !u0 || !u || threads < 1) return -1;
  const int m = n + 2;
  if (threads > n) threads = n;
  if (u != u0) memcpy(u, u0, sizeof(double) * (size_t)m * m);
  double *g = NULL;
  if (f) {
    const double h = 1.0 / (double)(n + 1);
    const double h2 = h * h;
    g = (double *)calloc((size_t)m * m, sizeof(double));
    if (!g) return -1;
    for (int i = 1; i <= n; ++i)
      for (int j = 1; j <= n; ++j) AT(g, i, j, m) = h2 * f[(size_t)(i - 1) * n + (j - 1)];
  }
  shared_t s;
  memset(&s, 0, sizeof(s));
  s.n = n;
  s.max_iters = max_iters;
  s.check_every = check_every;
  s.nthreads = threads;
  s.omega = omega;
  s.tol = tol;
  s.u = u;
  s.g = g;
  s.tmax = (double *)calloc((size_t)threads, sizeof(double));
  worker_t *ws = (worker_t *)calloc((size_t)threads, sizeof(worker_t));
  pthread_t *th = (pthread_t *)calloc((size_t)threads, sizeof(pthread_t));
  int rc = -1;
  pthread_mutex_init(&s.mu, NULL);
  pthread_cond_init(&s.cv, NULL);
  if (s.tmax && ws && th && pthread_barrier_init(&s.bar, NULL, (unsigned)threads) == 0) {
    int started = 0;
    for (int t = 0; t < threads; ++t) {
      ws[t].s = &s;
      ws[t].t = t;
      ws[t].i0 = 1 + (int)((long long)t * n / threads);
      ws[t].i1 = 1 + (int)((long long)(t + 1) * n / threads);
    }
    /* threads 1.. are created first and wait at the gate; the caller runs
     * thread 0's share once all exist (or releases them to exit) */
    rc = 0;
    for (int t = 1; t < threads; ++t) {
      if (pthread_create(&th[t], NULL, worker, &ws[t]) != 0) {
        rc = -1;
        break;
      }
      ++started;
    }
    pthread_mutex_lock(&s.mu);
    s.gate = rc == 0 ? 1 : -1;
    pthread_cond_broadcast(&s.cv);
    pthread_mutex_unlock(&s.mu);
    if (rc == 0) worker(&ws[0]);
    for (int t = 1; t <= started; ++t) pthread_join(th[t], NULL);
    pthread_barrier_destroy(&s.bar);
  }
  pthread_cond_destroy(&s.cv);
  pthread_mutex_destroy(&s.mu);
  free(th);
  free(ws);
  free(s.tmax);
  free(g);
  if (rc != 0) return -1;
  if (iterations) *iterations = s.iters;
  if (converged) *converged = s.conv;
  if (final_maxdelta) *final_maxdelta = s.mk;
  return 0;
}
