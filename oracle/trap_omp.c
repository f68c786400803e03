/* CPU multi-core baseline of the level-0 trapezoid kick -- TIMING INFRASTRUCTURE, NOT THE ORACLE.
 *
 * Like the oracle beside it, this file is test and benchmark infrastructure: the benchmark's CPU
 * baseline times it on all host cores as the multi-core CPU reference point for the GPU kick, and
 * a CPU test checks it against the oracle's trapezoid accelerations.  No parity claim rests on
 * it and the GPU library never calls it.
 *
 * It computes the accelerations of Sec. 2's pair loop over the right-angled trapezoid
 * (i = 0..N_m-1, j = i+1..N-1; a pair of the sorted flagged list weighted by g_0(r), the order-l
 * smooth step of the pair's position between the shell radii R_1 and R_0 (Sec. 3: R_0 from the
 * Hill radii, R_0 / R_1 the shell ratio), every other pair by 1; a dead body takes part in no
 * pair), with the trapezoid's rows shared among OpenMP threads.  Rows shorten as i grows, so the
 * rows are handed out dynamically in chunks; every thread sums into its own N x 3 array (a row
 * scatters into every j), and the arrays are added in thread order.  The per-pair arithmetic is
 * the oracle's, the order of the sums is not, so the two agree to rounding, not to the bit.
 */
#include <math.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* f_l(x) = x^{l+1} sum_{k=0}^{l} C(l+k, k) C(2l+1, l-k) (-x)^k on [0, 1], 0 below, 1 above */
static double smooth_step(double x, int l) {
  if (x <= 0.0) return 0.0;
  if (x >= 1.0) return 1.0;
  double s = 0.0, xk = 1.0;
  for (int k = 0; k <= l; ++k) {
    double c1 = 1.0, c2 = 1.0;
    for (int i = 1; i <= k; ++i) c1 = c1 * (double)(l + i) / (double)i;            /* C(l+k, k) */
    for (int i = 1; i <= l - k; ++i) c2 = c2 * (double)(l + k + 1 + i) / (double)i; /* C(2l+1, l-k) */
    s += c1 * c2 * xk;
    xk *= -x;
  }
  double xp = 1.0;
  for (int k = 0; k <= l; ++k) xp *= x;
  return xp * s;
}

/* Returns the number of threads used (>= 1), or -1 when scratch memory could not be allocated.
 * x: 3n interleaved positions; a: 3n accelerations (out); pairs: 2 npairs, sorted by (i, j), i < j.
 * threads <= 0: every thread OpenMP offers. */
int trap_omp_accel(int n, int n_massive, const double *x, const double *m, const double *rhill,
                   const int *alive, const int *pairs, int npairs, double G, double hill_scale,
                   double shell_ratio, int l, int threads, double *a) {
  int T = 1;
#ifdef _OPENMP
  T = threads > 0 ? threads : omp_get_max_threads();
#endif
  if (T < 1) T = 1;
  int *row = (int *)malloc(sizeof(int) * (size_t)(n_massive + 1));
  double *part = (double *)calloc((size_t)T * 3 * (size_t)n, sizeof(double));
  if (!row || !part) {
    free(row);
    free(part);
    return -1;
  }
  /* row[i]: first flagged pair of row i (the list is sorted) */
  for (int i = 0, q = 0; i <= n_massive; ++i) {
    while (q < npairs && pairs[2 * q] < i) ++q;
    row[i] = q;
  }
#ifdef _OPENMP
#pragma omp parallel for num_threads(T) schedule(dynamic, 8)
#endif
  for (int i = 0; i < n_massive; ++i) {
    int t = 0;
#ifdef _OPENMP
    t = omp_get_thread_num();
#endif
    double *acc = part + (size_t)t * 3 * (size_t)n;
    if (!alive[i]) continue;
    int q = row[i];
    const int qend = row[i + 1];
    const double xi = x[3 * i], yi = x[3 * i + 1], zi = x[3 * i + 2];
    const double Gmi = G * m[i];
    double ax = 0.0, ay = 0.0, az = 0.0;
    for (int j = i + 1; j < n; ++j) {
      int flagged = 0;
      if (q < qend && pairs[2 * q + 1] == j) { flagged = 1; ++q; }
      if (!alive[j]) continue;
      const double dx = x[3 * j] - xi, dy = x[3 * j + 1] - yi, dz = x[3 * j + 2] - zi;
      const double r2 = (dx * dx + dy * dy) + dz * dz;
      const double r = sqrt(r2);
      const double r3 = r2 * r;
      double w = 1.0;
      if (flagged) {
        const double R0 = hill_scale * (rhill[i] + rhill[j]);
        const double R1 = R0 / shell_ratio;
        w = smooth_step((r - R1) / (R0 - R1), l);
      }
      const double fi = ((G * m[j]) * w) / r3;
      const double fj = (Gmi * w) / r3;
      ax += fi * dx;
      ay += fi * dy;
      az += fi * dz;
      acc[3 * j] -= fj * dx;
      acc[3 * j + 1] -= fj * dy;
      acc[3 * j + 2] -= fj * dz;
    }
    acc[3 * i] += ax;
    acc[3 * i + 1] += ay;
    acc[3 * i + 2] += az;
  }
#ifdef _OPENMP
#pragma omp parallel for num_threads(T) schedule(static)
#endif
  for (long k = 0; k < 3L * n; ++k) {
    double s = 0.0;
    for (int t = 0; t < T; ++t) s += part[(size_t)t * 3 * (size_t)n + (size_t)k];
    a[k] = s;
  }
  free(row);
  free(part);
  return T;
}
