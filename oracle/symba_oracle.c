/*
 * SyMBA oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, serial, FP64 CPU restatement of one SyMBA step (Duncan, Levison & Lee 1998, AJ 116,
 * 2067) with the SyMBAp parallel structure of Lau & Lee, arXiv:2304.07325:
 *   - every interaction of the right-angled trapezoid i < N_m, j > i  (Sec. 2, the nested loop);
 *   - close-encounter pairs grouped into independent groups that are integrated separately
 *     (Sec. 2, the GENGA-style grouping paragraph);
 *   - multiple time steps with subdivision factor M, shell ratio R_k/R_{k+1} and the partition
 *     function f_l with l = 3 (Sec. 3, first paragraph).
 * Where the paper only cites the method, the step follows the published SyMBA operator split
 * (democratic-heliocentric: sun drift / interaction kick / Kepler drift) and Danby's f and g
 * functions (Danby 1988, Fundamentals of Celestial Mechanics, Sec. 6.8).
 *
 * Only the test suite, the package smoke check and the benchmark's CPU-baseline leg may load this
 * library.  It shares no code, header, table or constant with the CUDA path.  It is deliberately
 * slow: no blocking, no fusion, no reordering beyond what the definitions state.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fno-fast-math -fPIC -shared symba_oracle.c -lm
 * (-ffp-contract=off matters: the encounter predicate and the sun drift are specified operation by
 * operation in IEEE round-to-nearest FP64, and gcc contracts a*b+c into an FMA on aarch64 by
 * default.)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_E_INVAL (-1)
#define ORC_E_NOMEM (-2)
#define ORC_E_KEPLER (-4)
#define ORC_E_DEPTH (-5)
#define ORC_E_NONFINITE (-7)
#define ORC_MAX_LEVELS 64

typedef struct {
  double dt;           /* tau: the full step */
  double shell_ratio;  /* R_k / R_{k+1} (2.08 in Sec. 3) */
  double hill_scale;   /* lambda: R_0^{ij} = lambda (rH_i + rH_j)  (reading; SWIFT-SyMBA uses 6.5) */
  double G;            /* gravitational constant (4 pi^2 in AU, yr, Msun) */
  double m0;           /* central mass */
  int M;               /* time-step subdivision factor (4 in Sec. 3) */
  int l;               /* order of the partition function f_l (3 in Sec. 3) */
  int max_depth;       /* deepest recursion level allowed */
  int noise;           /* test hook, 0 in every reference run: when set, each position and
                          velocity component a recursion sub-step kicks or drifts is multiplied by
                          1 +- 2^-52 (deterministic pseudo-random sign), to measure how strongly
                          the chaotic close encounters amplify differences at the rounding level */
  double rmin;         /* removal (reading; the paper names no rule): after the closing kick a  */
  double rmax;         /* live body with heliocentric r < rmin (the star) or r > rmax (ejected)  */
                       /* leaves the system; 0 switches a limit off */
} orc_params;

typedef struct {
  int n;               /* particles */
  int n_massive;       /* N_m: indices 0..N_m-1 are massive, N_m..n-1 are field particles */
  double *x;           /* [n][3] heliocentric positions */
  double *v;           /* [n][3] barycentric velocities (democratic heliocentric momenta / m) */
  double *m;           /* [n] masses (0 for field particles) */
  double *radius;      /* [n] physical radii (contact detection only) */
  double *rhill;       /* [n] Hill radii, fixed at init (rescaled when a body grows by a merger) */
  int *alive;          /* [n] 1 = in the system, 0 = merged into another body */
  int cap;             /* capacity of the output pair list below */
  int npairs;          /* level-0 encounter pairs found in the last step (may exceed cap) */
  int ngroups;         /* encounter groups in the last step */
  int *pairs;          /* [cap][2] level-0 pairs (i, j), i < j, in ascending (i, j) order */
  int *group_of_pair;  /* [cap] group index of each pair; groups are numbered by ascending label */
  int status;          /* worst status of the last step (0 = OK) */
  int max_depth_seen;  /* deepest level entered in the last step */
  long long collisions;            /* mergers (separation < R_i + R_j at a check) in the last step */
  long long removals;              /* bodies removed by rmin / rmax in the last step */
  long long level_flags[ORC_MAX_LEVELS]; /* pairs flagged at each level, summed over sub-steps */
  long long level_calls[ORC_MAX_LEVELS]; /* sub-steps E_k taken at each level in the last step */
} orc_sim;

/* ------------------------------------------------------------------------------------------ */
/* Correctly rounded summation.                                                                 */
/* The sum of a list of doubles, computed exactly and rounded once to nearest-even, using       */
/* Shewchuk's non-overlapping partials (Shewchuk 1997, "Adaptive precision floating-point       */
/* arithmetic and fast robust geometric predicates").  Every O(N) sum of the step (total        */
/* momentum, total mass) and the energy use it, so their value is a plain definition: the       */
/* exact sum of the listed terms, rounded once.                                                 */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
  double *p;
  long np, cap;
  double special; /* sum of non-finite inputs, if any */
  int nonfinite;
  int oom;
} orc_acc;

static void acc_init(orc_acc *a) {
  a->cap = 32;
  a->np = 0;
  a->p = (double *)malloc(sizeof(double) * (size_t)a->cap);
  a->special = 0.0;
  a->nonfinite = 0;
  a->oom = (a->p == NULL);
}

static void acc_free(orc_acc *a) { free(a->p); a->p = NULL; }

static void acc_add(orc_acc *a, double x) {
  if (a->oom) return;
  if (!isfinite(x)) { a->nonfinite = 1; a->special += x; return; }
  long i = 0;
  for (long k = 0; k < a->np; ++k) {
    double y = a->p[k];
    if (fabs(x) < fabs(y)) { double t = x; x = y; y = t; }
    double hi = x + y;
    double lo = y - (hi - x);
    if (lo != 0.0) a->p[i++] = lo;
    x = hi;
  }
  if (i >= a->cap) {
    long nc = a->cap * 2;
    double *q = (double *)realloc(a->p, sizeof(double) * (size_t)nc);
    if (!q) { a->oom = 1; return; }
    a->p = q; a->cap = nc;
  }
  a->p[i] = x;
  a->np = i + 1;
}

static double acc_result(const orc_acc *a) {
  if (a->nonfinite) return a->special;
  if (a->np == 0) return 0.0;
  long j = a->np - 1;
  double hi = a->p[j], lo = 0.0;
  while (j > 0) {
    double x = hi, y = a->p[--j];
    hi = x + y;
    double yr = hi - x;
    lo = y - yr;
    if (lo != 0.0) break;
  }
  /* half-way case: the partials below decide the direction of the tie */
  if (j > 0 && ((lo < 0.0 && a->p[j - 1] < 0.0) || (lo > 0.0 && a->p[j - 1] > 0.0))) {
    double y = lo * 2.0;
    double x = hi + y;
    double yr = x - hi;
    if (y == yr) hi = x;
  }
  return hi;
}

double orc_fsum(const double *a, long n) {
  orc_acc acc;
  acc_init(&acc);
  for (long k = 0; k < n; ++k) acc_add(&acc, a[k]);
  double r = acc_result(&acc);
  acc_free(&acc);
  return r;
}

/* ------------------------------------------------------------------------------------------ */
/* Partition (changeover) function f_l, Sec. 3 (l = 3 instead of the original l = 1).         */
/* Reading: f_l is the polynomial of degree 2l+1 rising from 0 at x = 0 to 1 at x = 1 with its  */
/* first l derivatives zero at both ends:                                                       */
/*   f_l(x) = x^{l+1} sum_{k=0}^{l} C(l+k, k) C(2l+1, l-k) (-x)^k,  clamped outside [0, 1].      */
/* l = 1 gives 3x^2 - 2x^3; l = 3 gives x^4 (35 - 84x + 70x^2 - 20x^3).                        */
/* ------------------------------------------------------------------------------------------ */
static double binom(int n, int k) {
  double r = 1.0;
  for (int i = 1; i <= k; ++i) r = r * (double)(n - k + i) / (double)i;
  return r;
}

double orc_partition(double x, int l) {
  if (x <= 0.0) return 0.0;
  if (x >= 1.0) return 1.0;
  double s = 0.0, xk = 1.0;
  for (int k = 0; k <= l; ++k) {
    s += binom(l + k, k) * binom(2 * l + 1, l - k) * xk;
    xk *= -x;
  }
  double xp = 1.0;
  for (int k = 0; k <= l; ++k) xp *= x;
  return xp * s;
}

/* Shell radii of a pair (reading of Duncan et al. 1998 Sec. 4): R_0 = lambda (rH_i + rH_j) and  */
/* R_k = R_0 c_k with c_0 = 1, c_k = c_{k-1} / (R_k/R_{k+1}).                                    */
static double shell_factor(const orc_params *P, int k) {
  double c = 1.0;
  for (int i = 0; i < k; ++i) c = c / P->shell_ratio;
  return c;
}

static double shell_R0(const orc_params *P, const orc_sim *s, int i, int j) {
  return P->hill_scale * (s->rhill[i] + s->rhill[j]);
}

/* g_k(r): 1 outside R_k, 0 inside R_{k+1}, f_l in between (g_k is the share of the pair       */
/* potential that stays at levels <= k).                                                        */
static double g_level(const orc_params *P, double R0, int k, double r) {
  double Rk = R0 * shell_factor(P, k);
  double Rk1 = R0 * shell_factor(P, k + 1);
  return orc_partition((r - Rk1) / (Rk - Rk1), P->l);
}

/* Weight of the pair force integrated at level k: w_0 = g_0, w_k = g_k - g_{k-1} (k >= 1).     */
/* The weights telescope: w_0 + ... + w_K = g_K, which tends to 1 as K grows.                  */
double orc_weight(const orc_params *P, double R0, int k, double r) {
  if (k == 0) return g_level(P, R0, 0, r);
  return g_level(P, R0, k, r) - g_level(P, R0, k - 1, r);
}

/* ------------------------------------------------------------------------------------------ */
/* Close-encounter predicate over an interval h with critical radius R (Sec. 2 gives the        */
/* concept; the geometry is the reading: linear relative motion over the interval).             */
/* Every operation is one IEEE FP64 operation in the order written.  Returns 1 if the pair is   */
/* flagged.  *contact is set if the same minimum distance is below Rc = R_i + R_j.              */
/* ------------------------------------------------------------------------------------------ */
int orc_encounter(const double *xi, const double *xj, const double *vi, const double *vj,
                  double R, double Rc, double h, int *contact) {
  double dx = xj[0] - xi[0], dy = xj[1] - xi[1], dz = xj[2] - xi[2];
  double dvx = vj[0] - vi[0], dvy = vj[1] - vi[1], dvz = vj[2] - vi[2];
  double r2 = (dx * dx + dy * dy) + dz * dz;
  double v2 = (dvx * dvx + dvy * dvy) + dvz * dvz;
  double vr = (dx * dvx + dy * dvy) + dz * dvz;
  double R2 = R * R;
  int flag;
  double dmin2;
  if (vr >= 0.0) {
    dmin2 = r2;
  } else {
    double t = -vr / v2;
    if (t < h) dmin2 = r2 - (vr * vr) / v2;
    else dmin2 = r2 + h * (2.0 * vr + h * v2);
  }
  if (r2 < R2) flag = 1;
  else if (vr >= 0.0) flag = 0;
  else flag = dmin2 < R2;
  *contact = 0;
  if (flag) {
    double Rc2 = Rc * Rc;
    *contact = dmin2 < Rc2;
  }
  return flag;
}

/* ------------------------------------------------------------------------------------------ */
/* Kepler drift: x, v advanced by dt on the two-body orbit of gravitational parameter mu,       */
/* with Danby's f and g functions.  Elliptic case (alpha > 0) in eccentric-anomaly difference;  */
/* alpha <= 0 in universal variables with Stumpff functions.  Returns ORC_OK or ORC_E_KEPLER.   */
/* The new state is x0 + ((f - 1) x0 + g v0), v0 + (f' x0 + (g' - 1) v0): over the short        */
/* intervals deep in the recursion f - 1 and g' - 1 (about -mu dt^2 / (2 r^3)) fall below half  */
/* an ulp of 1, so f and g' formed as 1 + (...) would round to 1 and lose them at every call.   */
/* ------------------------------------------------------------------------------------------ */

/* X - sin X without cancellation: its Taylor series for |X| < 1/2 (terms to X^23, the next    */
/* below 2^-60 of the first), X - sin X directly beyond.                                         */
static double x_minus_sin(double X) {
  if (fabs(X) >= 0.5) return X - sin(X);
  double X2 = X * X, term = X * X2 / 6.0, s = 0.0;
  for (int k = 1; k <= 11; ++k) {
    s += term;
    term *= -X2 / ((double)(2 * k + 2) * (double)(2 * k + 3));
  }
  return s;
}

static int drift_elliptic(double mu, double dt, double *x, double *v, double r0, double u,
                          double alpha) {
  double a = mu / alpha;
  double n = sqrt(mu / (a * a * a));
  double ec = 1.0 - r0 / a;        /* e cos E0 */
  double es = u / (n * a * a);     /* e sin E0 */
  double ndt = n * dt;
  /* f(X) = X - ec sin X + es (1 - cos X) - n dt is increasing (f' = r/a > 0) and its root lies  */
  /* within 2e of n dt; safeguarded Newton inside that bracket.                                  */
  double lo = ndt - 2.5, hi = ndt + 2.5;
  double X = ndt;
  int ok = 0;
  for (int it = 0; it < 200; ++it) {
    double sx = sin(X), sh = sin(0.5 * X);
    double omc = 2.0 * sh * sh; /* 1 - cos X */
    double fx = X - ec * sx + es * omc - ndt;
    double fp = 1.0 - ec * (1.0 - omc) + es * sx;
    if (fx > 0.0) hi = X; else lo = X;
    double dX = -fx / fp;
    double Xn = X + dX;
    if (fabs(dX) <= 1e-15 * fmax(1.0, fabs(X))) { X = Xn; ok = 1; break; }
    if (!(Xn > lo && Xn < hi)) Xn = 0.5 * (lo + hi);
    X = Xn;
  }
  if (!ok) return ORC_E_KEPLER;
  double sx = sin(X), sh = sin(0.5 * X);
  double omc = 2.0 * sh * sh;
  double r = a * (1.0 - ec * (1.0 - omc) + es * sx);
  double fm1 = -(a / r0) * omc;
  double g = dt - x_minus_sin(X) / n;
  double fdot = -(a * a * n * sx) / (r * r0);
  double gdm1 = -(a / r) * omc;
  double x0[3] = {x[0], x[1], x[2]}, v0[3] = {v[0], v[1], v[2]};
  for (int c = 0; c < 3; ++c) {
    x[c] = x0[c] + (fm1 * x0[c] + g * v0[c]);
    v[c] = v0[c] + (fdot * x0[c] + gdm1 * v0[c]);
  }
  return ORC_OK;
}

/* Stumpff functions c_k(z) for k = 0..3 (Danby 1988 Sec. 6.9). */
static void stumpff(double z, double c[4]) {
  if (fabs(z) < 0.1) {
    /* c_k(z) = sum_j (-z)^j / (2j + k)!  */
    for (int k = 0; k < 4; ++k) {
      double term = 1.0, s = 0.0;
      for (int i = 1; i <= k; ++i) term /= (double)i;
      for (int j = 0; j < 30; ++j) {
        s += term;
        term *= -z / ((double)(2 * j + k + 1) * (double)(2 * j + k + 2));
      }
      c[k] = s;
    }
    return;
  }
  if (z > 0.0) {
    double sz = sqrt(z);
    c[0] = cos(sz);
    c[1] = sin(sz) / sz;
  } else {
    double sz = sqrt(-z);
    c[0] = cosh(sz);
    c[1] = sinh(sz) / sz;
  }
  c[2] = (1.0 - c[0]) / z;
  c[3] = (1.0 - c[1]) / z;
}

static int drift_universal(double mu, double dt, double *x, double *v, double r0, double u,
                           double alpha) {
  /* Universal Kepler equation F(s) = r0 G1 + u G2 + mu G3 - dt with G_k = s^k c_k(alpha s^2); */
  /* F'(s) = r(s) > 0.  Safeguarded Newton on a bracket found by doubling.                      */
  double c[4];
  double sgn = dt >= 0.0 ? 1.0 : -1.0;
  double lo = 0.0, hi = fabs(dt) / r0;
  if (hi == 0.0) return ORC_OK;
  for (int it = 0; it < 200; ++it) {
    double s = sgn * hi;
    stumpff(alpha * s * s, c);
    double F = r0 * s * c[1] + u * s * s * c[2] + mu * s * s * s * c[3] - dt;
    if (sgn * F >= 0.0) break;
    lo = hi;
    hi *= 2.0;
    if (it == 199) return ORC_E_KEPLER;
  }
  double sa = 0.5 * (lo + hi);
  int ok = 0;
  for (int it = 0; it < 400; ++it) {
    double s = sgn * sa;
    stumpff(alpha * s * s, c);
    double G1 = s * c[1], G2 = s * s * c[2], G3 = s * s * s * c[3];
    double F = r0 * G1 + u * G2 + mu * G3 - dt;
    double Fp = r0 * c[0] + u * G1 + mu * G2;
    if (sgn * F > 0.0) hi = sa; else lo = sa;
    double ds = -F / Fp;
    double sn = sa + sgn * ds;
    if (fabs(ds) <= 1e-15 * fmax(1e-300, fabs(sa))) { sa = sn; ok = 1; break; }
    if (!(sn > lo && sn < hi)) sn = 0.5 * (lo + hi);
    sa = sn;
  }
  if (!ok) return ORC_E_KEPLER;
  double s = sgn * sa;
  stumpff(alpha * s * s, c);
  double G1 = s * c[1], G2 = s * s * c[2], G3 = s * s * s * c[3];
  double r = r0 * c[0] + u * G1 + mu * G2;
  double fm1 = -mu * G2 / r0;
  double g = dt - mu * G3;
  double fdot = -mu * G1 / (r * r0);
  double gdm1 = -mu * G2 / r;
  double x0[3] = {x[0], x[1], x[2]}, v0[3] = {v[0], v[1], v[2]};
  for (int k = 0; k < 3; ++k) {
    x[k] = x0[k] + (fm1 * x0[k] + g * v0[k]);
    v[k] = v0[k] + (fdot * x0[k] + gdm1 * v0[k]);
  }
  return ORC_OK;
}

int orc_kepler_drift(double mu, double dt, double *x, double *v) {
  double r0 = sqrt((x[0] * x[0] + x[1] * x[1]) + x[2] * x[2]);
  double v2 = (v[0] * v[0] + v[1] * v[1]) + v[2] * v[2];
  double u = (x[0] * v[0] + x[1] * v[1]) + x[2] * v[2];
  double alpha = 2.0 * mu / r0 - v2;
  if (!(r0 > 0.0) || !isfinite(alpha)) return ORC_E_NONFINITE;
  if (alpha > 0.0) return drift_elliptic(mu, dt, x, v, r0, u, alpha);
  return drift_universal(mu, dt, x, v, r0, u, alpha);
}

/* ------------------------------------------------------------------------------------------ */
/* Correctly rounded cube root: the double nearest the real cube root of x (IEEE 754-2008,     */
/* Sec. 9.2, lists it as rootn(x, 3)).  Hill radii (a (m / 3 m0)^{1/3}) and merged radii       */
/* ((R_i^3 + R_j^3)^{1/3}) are cube roots; libm's cbrt is only faithful, and one ulp of a      */
/* radius can decide a strict encounter or contact comparison at a tie, so the value used is   */
/* the one the definition fixes.                                                                */
/* Method: start from libm's candidate y and move it to the neighbouring double while x lies   */
/* outside y's rounding interval.  The cube is increasing, so y = RN(cbrt x) exactly when      */
/* b_lo^3 < x < b_hi^3, where b_lo and b_hi are the midpoints between y and its neighbours.    */
/* Each comparison is done on integers: b = B 2^k with B odd (54 bits), x = X 2^e, so          */
/* b^3 < x  <=>  B^3 < X 2^(e - 3k).  A midpoint's cube is never a double (B^3 is odd and has  */
/* more than 53 bits), so no comparison is a tie.                                               */
/* ------------------------------------------------------------------------------------------ */
#define MW 8 /* 8 x 32-bit words: 256 bits, more than the 165 a 55-bit cube or 53-bit x 2^t needs */

static void mw_from_u64(uint32_t a[MW], uint64_t v) {
  memset(a, 0, sizeof(uint32_t) * MW);
  a[0] = (uint32_t)v;
  a[1] = (uint32_t)(v >> 32);
}

/* r = a * b (schoolbook, words least significant first; the product must fit in MW words) */
static void mw_mul(uint32_t r[MW], const uint32_t a[MW], const uint32_t b[MW]) {
  uint32_t t[2 * MW];
  memset(t, 0, sizeof(t));
  for (int i = 0; i < MW; ++i) {
    uint64_t carry = 0;
    for (int j = 0; j < MW; ++j) {
      uint64_t cur = (uint64_t)a[i] * b[j] + t[i + j] + carry;
      t[i + j] = (uint32_t)cur;
      carry = cur >> 32;
    }
    t[i + MW] = (uint32_t)carry;
  }
  memcpy(r, t, sizeof(uint32_t) * MW);
}

/* r = v * 2^s */
static void mw_shl(uint32_t r[MW], uint64_t v, int s) {
  memset(r, 0, sizeof(uint32_t) * MW);
  for (int bit = 0; bit < 64; ++bit) {
    if ((v >> bit) & 1u) {
      int pos = bit + s;
      if (pos >= 0 && pos < 32 * MW) r[pos / 32] |= (uint32_t)1u << (pos % 32);
    }
  }
}

static int mw_cmp(const uint32_t a[MW], const uint32_t b[MW]) {
  for (int i = MW - 1; i >= 0; --i) {
    if (a[i] != b[i]) return a[i] < b[i] ? -1 : 1;
  }
  return 0;
}

/* sign of (B 2^k)^3 - X 2^e, for 2^53 - 1 <= B < 2^55 and 0 < X < 2^53 */
static int cube_minus(uint64_t B, int k, uint64_t X, int e) {
  int t = e - 3 * k;
  /* B^3 lies in [2^158, 2^165): X 2^t is below it for t < 0 and above it for t > 203 */
  if (t < 0) return 1;
  if (t > 32 * MW - 53) return -1;
  uint32_t b[MW], b2[MW], b3[MW], rhs[MW];
  mw_from_u64(b, B);
  mw_mul(b2, b, b);
  mw_mul(b3, b2, b);
  mw_shl(rhs, X, t);
  return mw_cmp(b3, rhs);
}

/* x = X 2^e with X an integer (x finite, positive) */
static void split_double(double x, uint64_t *X, int *e) {
  int ex;
  double f = frexp(x, &ex);            /* x = f 2^ex, f in [0.5, 1) */
  *X = (uint64_t)ldexp(f, 53);         /* exact: f has at most 53 significant bits */
  *e = ex - 53;
}

double orc_cbrt_rn(double x) {
  if (x == 0.0 || !isfinite(x)) return x;
  if (x < 0.0) return -orc_cbrt_rn(-x);
  uint64_t X;
  int e;
  split_double(x, &X, &e);
  double y = cbrt(x);
  for (int it = 0; it < 8; ++it) {
    uint64_t Y;
    int ey;
    split_double(y, &Y, &ey);          /* y = Y 2^ey, Y in [2^52, 2^53) (y is always normal) */
    /* upper boundary (y + next up) / 2 = (2Y + 1) 2^(ey - 1) */
    if (cube_minus(2 * Y + 1, ey - 1, X, e) < 0) { y = nextafter(y, INFINITY); continue; }
    /* lower boundary (next down + y) / 2: (2Y - 1) 2^(ey - 1), or (2^54 - 1) 2^(ey - 2) when y
       is a power of two (the spacing below it is half the spacing above) */
    uint64_t Bl = Y == (1ull << 52) ? (1ull << 54) - 1 : 2 * Y - 1;
    int kl = Y == (1ull << 52) ? ey - 2 : ey - 1;
    if (cube_minus(Bl, kl, X, e) > 0) { y = nextafter(y, 0.0); continue; }
    break;
  }
  return y;
}

/* ------------------------------------------------------------------------------------------ */
/* Democratic-heliocentric bookkeeping.                                                        */
/* ------------------------------------------------------------------------------------------ */

/* Total barycentric momentum P = sum_i m_i v_i, each component the correctly rounded sum of    */
/* the rounded products m_i * v_i,c.                                                            */
static void total_momentum(const orc_sim *s, double P[3]) {
  for (int c = 0; c < 3; ++c) {
    orc_acc a;
    acc_init(&a);
    for (int i = 0; i < s->n; ++i) acc_add(&a, s->m[i] * s->v[3 * i + c]);
    P[c] = acc_result(&a);
    acc_free(&a);
  }
}

/* Sun drift (the H_sun part of the split): x_i += h (P / m0), component by component:          */
/* q = P_c / m0, d = h * q, x = x + d.                                                          */
static void sun_drift(const orc_params *P, orc_sim *s, double h) {
  double Pt[3];
  total_momentum(s, Pt);
  for (int c = 0; c < 3; ++c) {
    double q = Pt[c] / P->m0;
    double d = h * q;
    for (int i = 0; i < s->n; ++i)
      if (s->alive[i]) s->x[3 * i + c] = s->x[3 * i + c] + d;
  }
}

/* Init: barycentric velocities v_i = v_i^hel - S / (m0 + Mt), with S = sum m_j v_j^hel and    */
/* Mt = sum m_j (both correctly rounded); Hill radii rH_i = a_i (m_i / (3 m0))^{1/3} with a_i  */
/* the osculating heliocentric semi-major axis for mu = G (m0 + m_i) (or r_i if unbound), from */
/* vis-viva 1/a = 2/r - v^2/mu; the cube root is the correctly rounded one (orc_cbrt_rn).       */
void orc_init(const orc_params *P, orc_sim *s, const double *v_helio, int compute_rhill) {
  orc_acc a;
  acc_init(&a);
  for (int i = 0; i < s->n; ++i) acc_add(&a, s->m[i]);
  double Mt = acc_result(&a);
  acc_free(&a);
  double denom = P->m0 + Mt;
  for (int c = 0; c < 3; ++c) {
    acc_init(&a);
    for (int i = 0; i < s->n; ++i) acc_add(&a, s->m[i] * v_helio[3 * i + c]);
    double S = acc_result(&a);
    acc_free(&a);
    double q = S / denom;
    for (int i = 0; i < s->n; ++i) s->v[3 * i + c] = v_helio[3 * i + c] - q;
  }
  if (compute_rhill) {
    for (int i = 0; i < s->n; ++i) {
      const double *xi = s->x + 3 * i, *vi = v_helio + 3 * i;
      double r = sqrt((xi[0] * xi[0] + xi[1] * xi[1]) + xi[2] * xi[2]);
      double v2 = (vi[0] * vi[0] + vi[1] * vi[1]) + vi[2] * vi[2];
      double mu = P->G * (P->m0 + s->m[i]);
      double inv_a = 2.0 / r - v2 / mu;
      double a_i = inv_a > 0.0 ? 1.0 / inv_a : r;
      s->rhill[i] = a_i * orc_cbrt_rn(s->m[i] / (3.0 * P->m0));
    }
  }
  s->status = ORC_OK;
}

/* Heliocentric velocities for output: v^hel_i = v_i + P / m0. */
void orc_velocity_helio(const orc_params *P, const orc_sim *s, double *v_helio) {
  double Pt[3];
  total_momentum(s, Pt);
  for (int c = 0; c < 3; ++c) {
    double q = Pt[c] / P->m0;
    for (int i = 0; i < s->n; ++i) v_helio[3 * i + c] = s->v[3 * i + c] + q;
  }
}

/* ------------------------------------------------------------------------------------------ */
/* Pair force and kicks.                                                                        */
/* The force of one pair at level k on i (and its reaction on j), in this operation order:      */
/*   d = x_j - x_i; r2 = (dx dx + dy dy) + dz dz; r = sqrt(r2); r3 = r2 r;                      */
/*   a_i += ((G m_j) w / r3) d;  a_j -= ((G m_i) w / r3) d.                                     */
/* ------------------------------------------------------------------------------------------ */
static void pair_accel(const orc_params *P, const orc_sim *s, int i, int j, int flagged, int k,
                       double *ai, double *aj) {
  const double *xi = s->x + 3 * i, *xj = s->x + 3 * j;
  double d[3] = {xj[0] - xi[0], xj[1] - xi[1], xj[2] - xi[2]};
  double r2 = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2];
  double r = sqrt(r2);
  double r3 = r2 * r;
  double w = 1.0;
  if (flagged) w = orc_weight(P, shell_R0(P, s, i, j), k, r);
  double fi = ((P->G * s->m[j]) * w) / r3;
  double fj = ((P->G * s->m[i]) * w) / r3;
  for (int c = 0; c < 3; ++c) {
    ai[c] += fi * d[c];
    aj[c] -= fj * d[c];
  }
}

/* Level-0 kick over the whole trapezoid (Sec. 2): i = 0..N_m-1, j = i+1..N-1.  Pairs in the     */
/* sorted flagged list use w_0 = g_0(r); all others w = 1.  Then v_i += h a_i.                  */
void orc_kick_trapezoid(const orc_params *P, orc_sim *s, const int *pairs, int npairs, double h) {
  double *a = (double *)calloc((size_t)s->n * 3, sizeof(double));
  int q = 0;
  for (int i = 0; i < s->n_massive; ++i) {
    for (int j = i + 1; j < s->n; ++j) {
      int flagged = 0;
      if (q < npairs && pairs[2 * q] == i && pairs[2 * q + 1] == j) { flagged = 1; ++q; }
      if (!s->alive[i] || !s->alive[j]) continue;
      pair_accel(P, s, i, j, flagged, 0, a + 3 * i, a + 3 * j);
    }
  }
  for (int i = 0; i < s->n; ++i) {
    if (!s->alive[i]) continue;
    for (int c = 0; c < 3; ++c) s->v[3 * i + c] = s->v[3 * i + c] + h * a[3 * i + c];
  }
  free(a);
}

/* Rounding-level perturbation of the sensitivity twin (see orc_params.noise): a SplitMix64 hash */
/* of (particle, component, counter) picks the sign.                                              */
static unsigned long long noise_counter = 0;

static double jiggle(double a, int p, int c) {
  unsigned long long z = (unsigned long long)p * 0x9E3779B97F4A7C15ull + (unsigned long long)c * 0xBF58476D1CE4E5B9ull +
                         (++noise_counter) * 0x94D049BB133111EBull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  const double eps = 2.220446049250313e-16;
  return a * (1.0 + ((z & 1ull) ? eps : -eps));
}

static void perturb(const orc_params *P, orc_sim *s, int p) {
  if (!P->noise) return;
  for (int c = 0; c < 3; ++c) {
    s->x[3 * p + c] = jiggle(s->x[3 * p + c], p, c);
    s->v[3 * p + c] = jiggle(s->v[3 * p + c], p, c + 3);
  }
}

/* Kick h over an explicit pair list at level k: accelerations summed pair by pair in list order, */
/* then v_p += h a_p once for every particle of the list.  `done` is an [n] scratch flag array.  */
static void kick_pairs(const orc_params *P, orc_sim *s, const int *pl, int np, int k, double h,
                       double *a, char *done) {
  for (int q = 0; q < 2 * np; ++q) {
    int p = pl[q];
    for (int c = 0; c < 3; ++c) a[3 * p + c] = 0.0;
    done[p] = 0;
  }
  for (int q = 0; q < np; ++q) {
    if (!s->alive[pl[2 * q]] || !s->alive[pl[2 * q + 1]]) continue;
    pair_accel(P, s, pl[2 * q], pl[2 * q + 1], 1, k, a + 3 * pl[2 * q], a + 3 * pl[2 * q + 1]);
  }
  for (int q = 0; q < 2 * np; ++q) {
    int p = pl[q];
    if (done[p] || !s->alive[p]) continue;
    for (int c = 0; c < 3; ++c) s->v[3 * p + c] = s->v[3 * p + c] + h * a[3 * p + c];
    perturb(P, s, p);
    done[p] = 1;
  }
}

/* ------------------------------------------------------------------------------------------ */
/* Grouping (Sec. 2): connected components of the graph whose edges are the flagged pairs.      */
/* Union-find; every component is labelled by its smallest particle index.                      */
/* ------------------------------------------------------------------------------------------ */
static int uf_find(int *parent, int x) {
  while (parent[x] != x) x = parent[x];
  return x;
}

void orc_union_find(int n, const int *pairs, int npairs, int *label) {
  for (int i = 0; i < n; ++i) label[i] = i;
  for (int q = 0; q < npairs; ++q) {
    int a = uf_find(label, pairs[2 * q]), b = uf_find(label, pairs[2 * q + 1]);
    if (a == b) continue;
    if (a < b) label[b] = a; else label[a] = b;
  }
  for (int i = 0; i < n; ++i) label[i] = uf_find(label, i);
}

/* ------------------------------------------------------------------------------------------ */
/* Merger on contact (reading: SyMBA merges colliding bodies; the paper's accuracy test reports  */
/* that none happened, which implies they can).  At a check of level k >= 1, a pair whose        */
/* current separation is below R_i + R_j merges: the lower index keeps the body with the summed */
/* mass, the mass-weighted position and barycentric velocity (momentum conserved), radius       */
/* (R_i^3 + R_j^3)^{1/3} and Hill radius rH_i (m / m_i)^{1/3}; the higher index leaves the      */
/* system (alive = 0, zero mass) and takes part in nothing afterwards.                          */
/* ------------------------------------------------------------------------------------------ */
static int in_contact(const orc_sim *s, int i, int j) {
  const double *xi = s->x + 3 * i, *xj = s->x + 3 * j;
  double dx = xj[0] - xi[0], dy = xj[1] - xi[1], dz = xj[2] - xi[2];
  double r2 = (dx * dx + dy * dy) + dz * dz;
  double Rc = s->radius[i] + s->radius[j];
  return r2 < Rc * Rc;
}

static void merge_pair(orc_sim *s, int i, int j) {
  double mi = s->m[i], mj = s->m[j];
  double M = mi + mj;
  if (M > 0.0) {
    for (int c = 0; c < 3; ++c) {
      s->x[3 * i + c] = (mi * s->x[3 * i + c] + mj * s->x[3 * j + c]) / M;
      s->v[3 * i + c] = (mi * s->v[3 * i + c] + mj * s->v[3 * j + c]) / M;
    }
  }
  double Ri = s->radius[i], Rj = s->radius[j];
  s->radius[i] = orc_cbrt_rn(Ri * Ri * Ri + Rj * Rj * Rj);
  if (mi > 0.0) s->rhill[i] = s->rhill[i] * orc_cbrt_rn(M / mi);
  s->m[i] = M;
  s->m[j] = 0.0;
  s->radius[j] = 0.0;
  s->rhill[j] = 0.0;
  s->alive[j] = 0;
  s->collisions++;
}

/* Removal: after the closing kick, a live body whose heliocentric distance is below rmin (it    */
/* has hit the star) or above rmax (it has been ejected) leaves the system like a body merged    */
/* away: mass, radii and flag zeroed, so the total momentum of the closing sun drift and of    */
/* every later sum no longer holds it.  r^2 = (x^2 + y^2) + z^2 against rmin^2 and rmax^2.      */
static void discard(const orc_params *P, orc_sim *s) {
  if (!(P->rmin > 0.0) && !(P->rmax > 0.0)) return;
  const double rmin2 = P->rmin * P->rmin, rmax2 = P->rmax * P->rmax;
  for (int i = 0; i < s->n; ++i) {
    if (!s->alive[i]) continue;
    const double *x = s->x + 3 * i;
    const double r2 = (x[0] * x[0] + x[1] * x[1]) + x[2] * x[2];
    if ((P->rmin > 0.0 && r2 < rmin2) || (P->rmax > 0.0 && r2 > rmax2)) {
      s->m[i] = 0.0;
      s->radius[i] = 0.0;
      s->rhill[i] = 0.0;
      s->alive[i] = 0;
      s->removals++;
    }
  }
}

/* ------------------------------------------------------------------------------------------ */
/* Recursive sub-stepping E_k(h) on one component, given its pairs F_{k-1} (sorted):            */
/*  (i)   F_k = pairs of F_{k-1} flagged at shell k over h;                                     */
/*  (ii)  kick h/2 over F_{k-1} with w_k;                                                        */
/*  (iii) particles of the component in no F_k pair: Kepler drift h; each component of F_k:     */
/*        M times E_{k+1}(h / M);                                                               */
/*  (iv)  kick h/2 over F_{k-1} with w_k.                                                        */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
  const orc_params *P;
  orc_sim *s;
  double *a;      /* [n][3] scratch accelerations */
  char *mark;     /* [n] scratch: drift bookkeeping */
  char *done;     /* [n] scratch: kick bookkeeping */
} orc_ctx;

static void E_level(orc_ctx *C, int k, double h, const int *F, int nF);

static void run_components(orc_ctx *C, int k, double h, const int *F, int nF) {
  /* components of the pair list F (labels = smallest index), each run as M x E_k(h) */
  orc_sim *s = C->s;
  int *lab = (int *)malloc(sizeof(int) * (size_t)s->n);
  /* union-find restricted to the particles of F */
  for (int q = 0; q < nF; ++q) { lab[F[2 * q]] = F[2 * q]; lab[F[2 * q + 1]] = F[2 * q + 1]; }
  for (int q = 0; q < nF; ++q) {
    int a = uf_find(lab, F[2 * q]), b = uf_find(lab, F[2 * q + 1]);
    if (a == b) continue;
    if (a < b) lab[b] = a; else lab[a] = b;
  }
  int *roots = (int *)malloc(sizeof(int) * (size_t)nF);
  int nroots = 0;
  for (int q = 0; q < nF; ++q) {
    int r = uf_find(lab, F[2 * q]);
    int seen = 0;
    for (int t = 0; t < nroots; ++t) if (roots[t] == r) seen = 1;
    if (!seen) roots[nroots++] = r;
  }
  /* ascending label order */
  for (int a = 1; a < nroots; ++a)
    for (int b = a; b > 0 && roots[b - 1] > roots[b]; --b) { int t = roots[b]; roots[b] = roots[b - 1]; roots[b - 1] = t; }
  int *sub = (int *)malloc(sizeof(int) * 2 * (size_t)nF);
  for (int t = 0; t < nroots; ++t) {
    int ns = 0;
    for (int q = 0; q < nF; ++q)
      if (uf_find(lab, F[2 * q]) == roots[t]) { sub[2 * ns] = F[2 * q]; sub[2 * ns + 1] = F[2 * q + 1]; ++ns; }
    for (int rep = 0; rep < C->P->M; ++rep) E_level(C, k, h, sub, ns);
  }
  free(sub);
  free(roots);
  free(lab);
}

static void E_level(orc_ctx *C, int k, double h, const int *F, int nF) {
  const orc_params *P = C->P;
  orc_sim *s = C->s;
  if (k > s->max_depth_seen) s->max_depth_seen = k;
  if (k < ORC_MAX_LEVELS) s->level_calls[k]++;
  /* (i) check F_{k-1} at shell k over h */
  int *Fk = (int *)malloc(sizeof(int) * 2 * (size_t)(nF > 0 ? nF : 1));
  int nk = 0;
  double ck = shell_factor(P, k);
  for (int q = 0; q < nF; ++q) {
    int i = F[2 * q], j = F[2 * q + 1], contact = 0;
    if (!s->alive[i] || !s->alive[j]) continue;
    if (in_contact(s, i, j)) { merge_pair(s, i, j); continue; }
    double Rk = shell_R0(P, s, i, j) * ck;
    double Rc = s->radius[i] + s->radius[j];
    if (orc_encounter(s->x + 3 * i, s->x + 3 * j, s->v + 3 * i, s->v + 3 * j, Rk, Rc, h, &contact)) {
      Fk[2 * nk] = i; Fk[2 * nk + 1] = j; ++nk;
    }
  }
  if (k < ORC_MAX_LEVELS) s->level_flags[k] += nk;
  double hh = 0.5 * h;
  /* (ii) */
  kick_pairs(P, s, F, nF, k, hh, C->a, C->done);
  /* (iii) */
  for (int q = 0; q < nF; ++q) { C->mark[F[2 * q]] = 0; C->mark[F[2 * q + 1]] = 0; }
  for (int q = 0; q < nk; ++q) { C->mark[Fk[2 * q]] = 1; C->mark[Fk[2 * q + 1]] = 1; }
  int deeper = nk > 0 && k + 1 <= P->max_depth;
  if (nk > 0 && !deeper && s->status == ORC_OK) s->status = ORC_E_DEPTH;
  double mu = P->G * P->m0;
  for (int q = 0; q < nF; ++q) {
    for (int e = 0; e < 2; ++e) {
      int p = F[2 * q + e];
      if (C->mark[p] == 1 && deeper) continue;
      if (C->mark[p] == 2 || !s->alive[p]) continue; /* already drifted, or merged away */
      int st = orc_kepler_drift(mu, h, s->x + 3 * p, s->v + 3 * p);
      if (st != ORC_OK && s->status == ORC_OK) s->status = st;
      perturb(P, s, p);
      C->mark[p] = 2;
    }
  }
  if (deeper) run_components(C, k + 1, h / (double)P->M, Fk, nk);
  /* (iv) */
  kick_pairs(P, s, F, nF, k, hh, C->a, C->done);
  free(Fk);
}

/* ------------------------------------------------------------------------------------------ */
/* One full step E(tau) (reading of the SyMBA split; parallel structure of Sec. 2):             */
/*  1. sun drift tau/2;                                                                         */
/*  2. level-0 check of every trapezoid pair over tau with R_0 -> flagged list F_0, groups;     */
/*  3. kick tau/2 (w_0 for flagged pairs);                                                      */
/*  4. Kepler drift tau for particles in no F_0 pair; each group: M times E_1(tau / M)          */
/*     (mergers happen inside these sub-steps);                                                 */
/*  5. kick tau/2 with the same F_0 at the new positions;                                       */
/*  6. sun drift tau/2.                                                                         */
/* ------------------------------------------------------------------------------------------ */
int orc_step(const orc_params *P, orc_sim *s) {
  if (!P || !s || s->n < 0 || s->n_massive < 0 || s->n_massive > s->n || P->M < 1)
    return ORC_E_INVAL;
  s->status = ORC_OK;
  s->max_depth_seen = 0;
  s->collisions = 0;
  s->removals = 0;
  for (int k = 0; k < ORC_MAX_LEVELS; ++k) { s->level_flags[k] = 0; s->level_calls[k] = 0; }
  const int n = s->n;
  const double tau = P->dt, half = 0.5 * tau;

  sun_drift(P, s, half);

  /* level-0 check, trapezoid order => the list comes out sorted by (i, j) */
  long capF = 64, nF = 0;
  int *F = (int *)malloc(sizeof(int) * 2 * (size_t)capF);
  if (!F) return ORC_E_NOMEM;
  for (int i = 0; i < s->n_massive; ++i) {
    if (!s->alive[i]) continue;
    for (int j = i + 1; j < n; ++j) {
      int contact = 0;
      if (!s->alive[j]) continue;
      double R0 = shell_R0(P, s, i, j);
      double Rc = s->radius[i] + s->radius[j];
      if (orc_encounter(s->x + 3 * i, s->x + 3 * j, s->v + 3 * i, s->v + 3 * j, R0, Rc, tau, &contact)) {
        if (nF == capF) {
          capF *= 2;
          int *G = (int *)realloc(F, sizeof(int) * 2 * (size_t)capF);
          if (!G) { free(F); return ORC_E_NOMEM; }
          F = G;
        }
        F[2 * nF] = i; F[2 * nF + 1] = j; ++nF;
      }
    }
  }
  s->level_flags[0] = nF;

  /* groups */
  int *label = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
  orc_union_find(n, F, (int)nF, label);
  char *inpair = (char *)calloc((size_t)(n > 0 ? n : 1), 1);
  for (long q = 0; q < nF; ++q) { inpair[F[2 * q]] = 1; inpair[F[2 * q + 1]] = 1; }
  int *gidx = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
  int ng = 0;
  for (int i = 0; i < n; ++i) gidx[i] = -1;
  for (int i = 0; i < n; ++i) if (inpair[i] && label[i] == i) gidx[i] = ng++;
  s->npairs = (int)nF;
  s->ngroups = ng;
  for (long q = 0; q < nF && q < s->cap; ++q) {
    s->pairs[2 * q] = F[2 * q];
    s->pairs[2 * q + 1] = F[2 * q + 1];
    s->group_of_pair[q] = gidx[label[F[2 * q]]];
  }

  orc_kick_trapezoid(P, s, F, (int)nF, half);

  double mu = P->G * P->m0;
  for (int i = 0; i < n; ++i) {
    if (inpair[i] || !s->alive[i]) continue;
    int st = orc_kepler_drift(mu, tau, s->x + 3 * i, s->v + 3 * i);
    if (st != ORC_OK && s->status == ORC_OK) s->status = st;
  }
  orc_ctx C;
  C.P = P; C.s = s;
  C.a = (double *)calloc((size_t)(n > 0 ? n : 1) * 3, sizeof(double));
  C.mark = (char *)calloc((size_t)(n > 0 ? n : 1), 1);
  C.done = (char *)calloc((size_t)(n > 0 ? n : 1), 1);
  if (nF > 0) run_components(&C, 1, tau / (double)P->M, F, (int)nF);

  orc_kick_trapezoid(P, s, F, (int)nF, half);
  discard(P, s);
  sun_drift(P, s, half);

  for (int i = 0; i < 3 * n; ++i)
    if (!isfinite(s->x[i]) || !isfinite(s->v[i])) { if (s->status == ORC_OK) s->status = ORC_E_NONFINITE; break; }

  free(C.a); free(C.mark); free(C.done); free(gidx); free(inpair); free(label); free(F);
  return s->status;
}

/* ------------------------------------------------------------------------------------------ */
/* Energy and angular momentum (democratic heliocentric; equal to the barycentric totals):       */
/*  E = sum_i (0.5 m_i) |v_i|^2 + |P|^2 / (2 m0) - sum_i (G m0) m_i / |x_i|                     */
/*      - sum_{trapezoid pairs} (G m_i) m_j / |x_j - x_i|                                       */
/*  L = sum_i m_i (x_i x v_i)                                                                    */
/* each the correctly rounded sum of its terms, every term in the operation order written.      */
/* ------------------------------------------------------------------------------------------ */
void orc_energy(const orc_params *P, const orc_sim *s, double *E, double *L) {
  double Pt[3];
  total_momentum(s, Pt);
  orc_acc a;
  acc_init(&a);
  const double Gm0 = P->G * P->m0;
  for (int i = 0; i < s->n; ++i) {
    if (!s->alive[i]) continue;
    const double *v = s->v + 3 * i, *x = s->x + 3 * i;
    double v2 = (v[0] * v[0] + v[1] * v[1]) + v[2] * v[2];
    acc_add(&a, (0.5 * s->m[i]) * v2);
    double r = sqrt((x[0] * x[0] + x[1] * x[1]) + x[2] * x[2]);
    acc_add(&a, -((Gm0 * s->m[i]) / r));
  }
  double P2 = (Pt[0] * Pt[0] + Pt[1] * Pt[1]) + Pt[2] * Pt[2];
  acc_add(&a, P2 / (2.0 * P->m0));
  for (int i = 0; i < s->n_massive; ++i) {
    if (!s->alive[i]) continue;
    const double *xi = s->x + 3 * i;
    double Gmi = P->G * s->m[i];
    for (int j = i + 1; j < s->n; ++j) {
      if (!s->alive[j]) continue;
      const double *xj = s->x + 3 * j;
      double dx = xj[0] - xi[0], dy = xj[1] - xi[1], dz = xj[2] - xi[2];
      double r = sqrt((dx * dx + dy * dy) + dz * dz);
      acc_add(&a, -((Gmi * s->m[j]) / r));
    }
  }
  *E = acc_result(&a);
  acc_free(&a);
  for (int c = 0; c < 3; ++c) {
    int c1 = (c + 1) % 3, c2 = (c + 2) % 3;
    acc_init(&a);
    for (int i = 0; i < s->n; ++i) {
      if (!s->alive[i]) continue;
      const double *x = s->x + 3 * i, *v = s->v + 3 * i;
      acc_add(&a, s->m[i] * (x[c1] * v[c2] - x[c2] * v[c1]));
    }
    L[c] = acc_result(&a);
    acc_free(&a);
  }
}

/* Accelerations of the level-0 trapezoid (all pairs w = 1 except the flagged list), without    */
/* touching the state: used by the tests to compare against brute force.                       */
void orc_accel_trapezoid(const orc_params *P, orc_sim *s, const int *pairs, int npairs, double *a) {
  for (int i = 0; i < 3 * s->n; ++i) a[i] = 0.0;
  int q = 0;
  for (int i = 0; i < s->n_massive; ++i)
    for (int j = i + 1; j < s->n; ++j) {
      int flagged = 0;
      if (q < npairs && pairs[2 * q] == i && pairs[2 * q + 1] == j) { flagged = 1; ++q; }
      if (!s->alive[i] || !s->alive[j]) continue;
      pair_accel(P, s, i, j, flagged, 0, a + 3 * i, a + 3 * j);
    }
}
