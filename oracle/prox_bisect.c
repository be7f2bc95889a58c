/*
 * Per-cell proximal map of tau*phi by bisection (Sec. 3; the scalar equation
 * is derived in oracle/prox.py from the first-order conditions for q' = 2).
 * Test infrastructure: part of the CPU oracle, never linked into the CUDA
 * library.
 *
 * This is the same algorithm as prox_cells in oracle/prox.py, written out per
 * cell in plain C so that full-size runs of the oracle finish in test time:
 *   P = P_K(w_bar) componentwise (signs +, -, +, -), |P|^2 summed in component
 *   order;
 *   h(m) = ((m - m_bar) + tau ((a m + (b m) m) + c)) - (tau |P|^2) / (2 (m + tau)^2);
 *   h(0) >= 0  ->  (m, w) = (0, 0);
 *   otherwise bisect [0, max(0, m_bar - tau c) + |P|^2/(2 tau)] with
 *   mid = lo + (hi - lo)/2 until mid equals an endpoint, keep the endpoint
 *   with the smaller |h|, and set w = m/(m + tau) P.
 * Every operation is a separately rounded IEEE double operation in the order
 * written (built with -ffp-contract=off), so the result equals the NumPy
 * version bit for bit; a CPU test checks that.
 */
#include <pthread.h>
#include <stddef.h>

static double h_eq(double m, double mbar, double P2, double tau, double a, double b, double c) {
  const double t = m + tau;
  return ((m - mbar) + tau * ((a * m + (b * m) * m) + c)) - (tau * P2) / (2.0 * (t * t));
}

static void prox_one(long long e, long long n, int nw, double tau, const double* v, const double* a,
                     double b, const double* c, double* out, int max_iter) {
  const double mbar = v[e];
  double P[4] = {0.0, 0.0, 0.0, 0.0};
  double P2 = 0.0;
  for (int q = 0; q < nw; ++q) {
    const double x = v[(long long)(q + 1) * n + e];
    /* clip like NumPy's maximum/minimum: the argument itself when it is on the
       kept side, equal to the bound, or NaN */
    if (q % 2 == 0)
      P[q] = (x >= 0.0 || x != x) ? x : 0.0;
    else
      P[q] = (x <= 0.0 || x != x) ? x : 0.0;
  }
  for (int q = 0; q < nw; ++q) P2 = (q == 0) ? P[0] * P[0] : P2 + P[q] * P[q];
  const double ae = a[e], ce = c[e];
  double m;
  const int zero = h_eq(0.0, mbar, P2, tau, ae, b, ce) >= 0.0;
  if (zero) {
    m = 0.0;
  } else {
    double lo = 0.0;
    const double t0 = mbar - tau * ce;
    double hi = (0.0 >= t0 ? 0.0 : t0) + P2 / (2.0 * tau); /* NumPy's maximum(0, t0) */
    for (int it = 0; it < max_iter; ++it) {
      const double mid = lo + 0.5 * (hi - lo);
      if (mid <= lo || mid >= hi) break;
      const double hm = h_eq(mid, mbar, P2, tau, ae, b, ce);
      if (hm < 0.0)
        lo = mid;
      else
        hi = mid;
    }
    double hlo = h_eq(lo, mbar, P2, tau, ae, b, ce);
    double hhi = h_eq(hi, mbar, P2, tau, ae, b, ce);
    hlo = hlo < 0.0 ? -hlo : hlo;
    hhi = hhi < 0.0 ? -hhi : hhi;
    m = (hlo < hhi) ? lo : hi;
  }
  out[e] = m;
  const double s = m / (m + tau);
  for (int q = 0; q < nw; ++q) out[(long long)(q + 1) * n + e] = zero ? 0.0 : s * P[q];
}

typedef struct {
  long long begin, end, n;
  int nw, max_iter;
  double tau, b;
  const double *v, *a, *c;
  double* out;
} job_t;

static void* run_job(void* arg) {
  const job_t* j = (const job_t*)arg;
  for (long long e = j->begin; e < j->end; ++e)
    prox_one(e, j->n, j->nw, j->tau, j->v, j->a, j->b, j->c, j->out, j->max_iter);
  return NULL;
}

/* v, out: (1 + nw) x n, component-major (m first); a, c: n; b scalar.
 * Cells are split into `nthreads` contiguous ranges, one thread each; every
 * cell is computed independently, so the result does not depend on the split. */
int oracle_prox_cells(int nw, long long n, double tau, const double* v, const double* a, double b,
                      const double* c, double* out, int max_iter, int nthreads) {
  if (nw < 0 || nw > 4 || n < 0) return 1;
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  if ((long long)nthreads > n) nthreads = n > 0 ? (int)n : 1;
  pthread_t th[256];
  int live[256];
  job_t jobs[256];
  const long long per = (n + nthreads - 1) / nthreads;
  for (int t = 0; t < nthreads; ++t) {
    live[t] = 0;
    jobs[t].begin = (long long)t * per < n ? (long long)t * per : n;
    jobs[t].end = jobs[t].begin + per < n ? jobs[t].begin + per : n;
    jobs[t].n = n;
    jobs[t].nw = nw;
    jobs[t].max_iter = max_iter;
    jobs[t].tau = tau;
    jobs[t].b = b;
    jobs[t].v = v;
    jobs[t].a = a;
    jobs[t].c = c;
    jobs[t].out = out;
    if (t == 0 || jobs[t].begin >= jobs[t].end) continue;
    if (pthread_create(&th[t], NULL, run_job, &jobs[t]) == 0)
      live[t] = 1;
    else
      run_job(&jobs[t]); /* no thread available: do the range here */
  }
  run_job(&jobs[0]);
  for (int t = 1; t < nthreads; ++t)
    if (live[t]) pthread_join(th[t], NULL);
  return 0;
}
