// Internal data layout and device helpers of the SyMBA GB300 path.
//
// Layout in HBM (all systems of a pool share the arrays; system d owns particles
// [off_d, off_d + n_d), off_d a multiple of 32):
//   x, y, z, vx, vy, vz, m, gm (= G m), rad, rh   : FP64 SoA, heliocentric x, barycentric v
//   alive, gid                                     : int per particle (gid = encounter group or -1)
//   xf, yf, zf, vxf, vyf, vzf, lamf, sigf          : FP32 copies for the encounter prefilter
//   tiles                                          : int4 {system, first row block, first column block,
//                                                    end of the massive blocks} per 4 x 4 macro-tile
//                                                    of 32 x 32 tiles (128-body quads q <= c)
//   fblk                                           : int2 {system, block} per block of field particles
//   part                                           : FP64 [macro-tile][rows, columns][4][3][32]
//                                                    pair-kick partials
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/symba.h"

#define SYM_TILE 32
#define SYM_MAX_LEVELS 32
#define SYM_PAIR_LC (16 * (SYM_MAX_LEVELS + 2))   // level-constant cache of one recursion warp
#define SYM_REC_BPSM_MAX 2   // recursion CTAs per SM a schedule may ask for
#define SA_NDIG 68  // 32-bit digits of the exact accumulator, digit k weighs 2^(32k - 1088)
#ifndef SYM_MACRO_COLS
#define SYM_MACRO_COLS 2     // column blocks of a macro-tile (its rows: 4 blocks, one per warp)
#endif
#define SYM_MACRO_PART ((4 + SYM_MACRO_COLS) * 96)   // partials of a macro-tile: rows, then columns,
                                                     // [block][3][32] each

struct DiskDesc {
  int off, n, nm, nb, nbm;      // first particle, counts, 32-blocks (all, massive rows)
  int tile_base, ntiles;        // this system's macro-tiles in the global list
  int pair_base, pair_cap;      // this system's slice of the pair buffers
  int group_base;               // this system's slice of the group slots (= off / 2)
  int active, M, l, max_depth, max_substeps, pad0;
  double dt, shell_ratio, hill_scale, G, m0;
  double rmin2, rmax2;          // squared removal distances (0 = no limit)
  double ck[SYM_MAX_LEVELS + 2];    // c_k = c_{k-1} / shell_ratio, c_0 = 1 (R_k = R_0 c_k)
  double ck2[SYM_MAX_LEVELS + 2];   // c_k^2
  double invdc[SYM_MAX_LEVELS + 2]; // 1 / (c_k - c_{k+1})
};

struct DiskStat {               // mutable per-system counters (device)
  int npairs, ngroups, status, max_depth;
  unsigned long long merges, substeps, merges_reported;
  unsigned long long max_chain;   // most sub-steps of one group in one step
  unsigned long long removals;    // bodies removed by rmin / rmax
  unsigned long long pair_substeps;   // sub-steps the single-pair path took
};

struct Dev {
  // particle SoA
  double *x, *y, *z, *vx, *vy, *vz, *m, *gm, *rad, *rh;
  int *alive, *gid;
  float *xf, *yf, *zf, *vxf, *vyf, *vzf, *lamf, *sigf;
  float *xl, *yl, *zl;          // low parts of positions (mixed precision: x = xf + xl)
  float *gmf;                   // G m in FP32 (mixed precision)
  int *blk_disk;                // system of each 32-block
  // systems
  DiskDesc *disks;
  DiskStat *stat;
  double *P;                    // [max_disks][3] total barycentric momentum (for the sun drift)
  unsigned long long *sacc;     // [max_disks][3][SA_NDIG + 1] exact accumulators
  // trapezoid
  int4 *tiles;                  // macro-tiles (quads q <= c) over the blocks holding massive bodies
  double *part;                 // [macro-tile][SYM_MACRO_PART]
  int2 *fblk;                   // field rectangle: {system, block} of every block of field particles only
  int nfblk;
  int *work;                    // [4] dynamic work counters (kick 1, kick 2, recursion, spare)
  int ntiles_total;
  int seg_len;                  // macro-tiles per work item
  int ndisks;                   // slots in use (upper bound of active slots)
  // encounter pairs (pair-indexed, per-system slices)
  int *raw_i, *raw_j;           // appended by the fused check, unordered
  int *pi, *pj, *gop;           // sorted (i, j) and group of each pair (local group index)
  int *gpi, *gpj;               // pairs grouped by group, sorted within a group (global indices)
  int *lev;                     // recursion level marks per grouped pair
  int *perm, *ptmp;             // nested active-pair lists of the recursion (per grouped pair)
  double *pR0, *pinvR0;         // level-0 critical radius of each grouped pair and its inverse
  int *mperm, *mtmp;            // nested active-member lists (per member slot)
  // member-slot copies of the bodies of large groups (indexed like gmem)
  double *gx, *gy, *gz, *gvx, *gvy, *gvz, *gmm, *ggm, *grad, *grh;
  int *galive;
  int *gpa, *gpb;               // grouped pair -> member slots (large groups)
  double *pf;                   // [pair][5] per-pair force scratch (d, fi, fj)
  int *adj;                     // [2 * pair] adjacency: (grouped pair index << 1) | side
  // particle-indexed scratch for grouping
  int *cnt, *start, *cursor, *parent, *inpair, *gidx, *tmpj, *mslot, *adj_off, *adj_cnt;
  double *acc;                  // [particle][3] recursion accelerations
  // groups (group slots, per-system slices)
  int *g_moff, *g_mcnt, *g_poff, *g_pcnt, *g_cur;
  int *gmem;                    // members grouped by group (global particle indices)
  int *rec_items;               // recursion work list (global group slot)
  int *rec_total;               // number of items
  double *lcache;               // [recursion warp][SYM_PAIR_LC] single-pair level constants
};

// --------------------------------------------------------------------------------------------
// small helpers
// --------------------------------------------------------------------------------------------
__device__ __forceinline__ void set_status(DiskStat *st, int code) {
  atomicCAS(&st->status, 0, code);
}

__device__ __forceinline__ int find_disk(const int *blk_disk, int p) { return blk_disk[p >> 5]; }

// The double nearest M 2^e2 (M > 0; ties away from zero), built on the integer pipe: normalise,
// keep 53 bits, add the rounding bit; adding the 53-bit significand (hidden bit included) to
// (exponent - 1) << 52 carries into the exponent field by itself.  Normal results only.
__device__ __forceinline__ double u64_scaled(unsigned long long M, int e2) {
  const int lz = __clzll(M);
  const unsigned long long n = M << lz;                       // top bit at 63
  const unsigned long long m = (n >> 11) + ((n >> 10) & 1ull);  // in [2^52, 2^53]
  const long long ex = (long long)(e2 - lz + 63 + 1022);
  return __longlong_as_double((long long)(((unsigned long long)ex << 52) + m));
}

// r^-3 for the pair kick with two FP64 instructions (the kick is bound by the FP64 pipe, so the
// rest of the work goes to the integer pipe and one MUFU operation):
//   seed     y0 = Y 2^ye (Y a 24-bit integer) from one MUFU rsqrt of the top 24 bits of r2,
//            |1 - r2 y0^2| < 2^-21;
//   Newton   one step in 64-bit integers: D = 2^k (1 - r2 y0^2) from the high word of R Y^2 (R
//            the 53-bit significand of r2), y1 = y0 (1 + (1 - r2 y0^2) / 2) kept as a ~40-bit
//            integer Y1 (|1 - r2 y1^2| < 2^-37);
//   powers   t = RN(y1^2), c = RN(y1^3), c15 = RN(3/2 y1^3) from Y1 on the integer pipe;
//   finish   e = 1 - r2 t (one FMA), r^-3 = y1^3 (1 - e)^{-3/2} = c + c15 e (one FMA; the next
//            term 15/8 e^2 < 2^-72 is far below the rounding).
// Error below 1.7 x 2^-52 relative (y1's quantisation enters only through e; t, c and the two
// FMAs round once each).  Values of r2 outside the normal FP32 range take the library path.
__device__ __forceinline__ double rinv3(double r2) {
  const unsigned long long rb = (unsigned long long)__double_as_longlong(r2);
  const int E = (int)(rb >> 52) & 0x7FF;
  const int fe = E - 896;
  if ((unsigned)(fe - 1) <= 253u && (long long)rb > 0) {
    const unsigned m23 = (unsigned)(rb >> 29) & 0x7FFFFFu;
    const float r2f = __uint_as_float(((unsigned)fe << 23) | m23);
    float y0f;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y0f) : "f"(r2f));
    const unsigned yb = __float_as_uint(y0f);
    const long long Y = (long long)((yb & 0x7FFFFFu) | 0x800000u);
    const int ye = (int)((yb >> 23) & 0xFFu) - 150;                        // y0 = Y 2^ye
    const unsigned long long R = (rb & 0xFFFFFFFFFFFFFull) | (1ull << 52);  // r2 = R 2^(E-1075)
    const unsigned long long H = __umul64hi(R << 11, (unsigned long long)(Y * Y) << 16);
    const int k = 1038 - E - 2 * ye;                  // R Y^2 2^-37 = H ~ 2^k, k in 61..64
    // D = 2^k - H, |D| < 2^(k-20); for k = 64 the unsigned difference wraps to 2^64 - H
    const long long D = (long long)((k < 64 ? (1ull << (k & 63)) : 0ull) - H);
    const long long Dp = k <= 63 ? (D << ((63 - k) & 63)) : (D >> 1);       // D 2^(63-k)
    const long long C = __mul64hi(Y << 16, Dp << 16) >> 16;                  // Y D' 2^-48
    const unsigned long long Y1 = (unsigned long long)((Y << 16) + C);       // y1 = Y1 2^(ye-16)
    const int sh = __clzll(Y1);
    const unsigned long long N = Y1 << sh;                                    // y1 = N 2^(ye-16-sh)
    const int ne = ye - 16 - sh;
    const unsigned long long Q = __umul64hi(N, N);                            // N^2 2^-64
    const unsigned long long QN = __umul64hi(Q, N);                           // N^3 2^-128
    const double t = u64_scaled(Q, 2 * ne + 64);
    const double c = u64_scaled(QN, 3 * ne + 128);
    const double c15 = u64_scaled(3ull * (QN >> 2), 3 * ne + 129);
    const double e = fma(-r2, t, 1.0);
    return fma(e, c15, c);
  }
  const double y = rsqrt(r2);
  return y * y * y;
}

// 1/sqrt(r2) to full FP64 accuracy: the same integer-built FP32 seed, then the third-order
// correction y = y0 (1 + e/2 + 3e^2/8), e = 1 - r2 y0^2 (5 FP64 instructions).
__device__ __forceinline__ double rsqrt_fp64(double r2) {
  const int hi = __double2hiint(r2);
  const unsigned lo = (unsigned)__double2loint(r2);
  const int fe = ((hi >> 20) & 0x7FF) - 896;
  if ((unsigned)(fe - 1) <= 253u && hi > 0) {
    const unsigned m23 = ((unsigned)(hi & 0xFFFFF) << 3) | (lo >> 29);
    const float r2f = __uint_as_float(((unsigned)fe << 23) | m23);
    float y0f;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y0f) : "f"(r2f));
    const unsigned yb = __float_as_uint(y0f);
    const int ye = (int)((yb >> 23) & 0xFF) + 896;
    const double y0 = __hiloint2double((ye << 20) | (int)((yb & 0x7FFFFF) >> 3), (int)((yb & 7u) << 29));
    const double e = fma(-r2, y0 * y0, 1.0);
    return fma(y0 * e, fma(e, 0.375, 0.5), y0);
  }
  return rsqrt(r2);
}

// Correctly rounded cube root: the double nearest the real cube root (IEEE 754-2008 Sec. 9.2,
// rootn(x, 3)).  Hill radii a (m / 3 m0)^{1/3} and merged radii (R_a^3 + R_b^3)^{1/3} are cube
// roots, and a radius feeds strict encounter and contact comparisons, so it takes the one value
// the definition fixes rather than the library's faithful (1-ulp) result.  The library value is
// the starting candidate y; since t -> t^3 is increasing, y is the nearest double exactly when
// x lies strictly between the cubes of y's rounding boundaries (the midpoints to its
// neighbours), and y moves one double up or down until it does.  A boundary is B 2^k with B an
// odd integer below 2^55 and x = X 2^e with X below 2^53, so b^3 < x  <=>  B^3 < X 2^(e - 3k),
// compared on 192-bit integers (three 64-bit words).  B^3 is odd with more than 53 significant
// bits, so it never equals X 2^(e - 3k): no ties.  Off the hot path (set-up and mergers).
struct U192 {
  unsigned long long w0, w1, w2;   // least significant first
};

__device__ __forceinline__ U192 cube_u192(unsigned long long B) {
  const unsigned long long s0 = B * B, s1 = __umul64hi(B, B);          // B^2 < 2^110
  const unsigned long long a0 = s0 * B, a1 = __umul64hi(s0, B);
  const unsigned long long b0 = s1 * B, b1 = __umul64hi(s1, B);
  U192 r;
  r.w0 = a0;
  r.w1 = a1 + b0;
  r.w2 = b1 + (r.w1 < a1 ? 1ull : 0ull);
  return r;
}

// sign of B^3 - X 2^t for 2^53 - 1 <= B < 2^55 (B^3 in [2^158, 2^165)) and 0 < X < 2^53
__device__ __forceinline__ int cube_cmp(unsigned long long B, unsigned long long X, int t) {
  if (t < 0) return 1;
  if (t > 192 - 53) return -1;
  U192 rhs = {0ull, 0ull, 0ull};
  const int q = t >> 6, s = t & 63;
  const unsigned long long lo = X << s, hi = s ? (X >> (64 - s)) : 0ull;
  if (q == 0) { rhs.w0 = lo; rhs.w1 = hi; }
  else if (q == 1) { rhs.w1 = lo; rhs.w2 = hi; }
  else { rhs.w2 = lo; }
  const U192 c = cube_u192(B);
  if (c.w2 != rhs.w2) return c.w2 < rhs.w2 ? -1 : 1;
  if (c.w1 != rhs.w1) return c.w1 < rhs.w1 ? -1 : 1;
  if (c.w0 != rhs.w0) return c.w0 < rhs.w0 ? -1 : 1;
  return 0;
}

static __device__ __noinline__ double cbrt_rn(double x) {
  if (x == 0.0 || !isfinite(x)) return x;
  const bool negative = x < 0.0;
  const double ax = fabs(x);
  const unsigned long long xb = (unsigned long long)__double_as_longlong(ax);
  const int xe = (int)(xb >> 52);
  const unsigned long long X = xe ? ((xb & 0xFFFFFFFFFFFFFull) | (1ull << 52)) : xb;
  const int e = (xe ? xe : 1) - 1075;                     // ax = X 2^e (subnormals included)
  double y = cbrt(ax);                                    // within one ulp; always normal
  for (int it = 0; it < 8; ++it) {
    const unsigned long long yb = (unsigned long long)__double_as_longlong(y);
    const unsigned long long Y = (yb & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const int ey = (int)(yb >> 52) - 1075;                // y = Y 2^ey
    // upper boundary (2Y + 1) 2^(ey - 1): below the root -> y is too small
    if (cube_cmp(2 * Y + 1, X, e - 3 * (ey - 1)) < 0) {
      y = __longlong_as_double((long long)(yb + 1));
      continue;
    }
    // lower boundary: (2Y - 1) 2^(ey - 1), or (2^54 - 1) 2^(ey - 2) below a power of two
    const bool pow2 = Y == (1ull << 52);
    const unsigned long long Bl = pow2 ? (1ull << 54) - 1 : 2 * Y - 1;
    const int kl = pow2 ? ey - 2 : ey - 1;
    if (cube_cmp(Bl, X, e - 3 * kl) > 0) {
      y = __longlong_as_double((long long)(yb - 1));
      continue;
    }
    break;
  }
  return negative ? -y : y;
}

// Order of non-negative doubles through their bit patterns (an integer comparison instead of an
// FP64-pipe one; valid for +0, finite and +inf operands).
__device__ __forceinline__ bool lt_nn(double a, double b) {
  return __double_as_longlong(a) < __double_as_longlong(b);
}
__device__ __forceinline__ bool is_neg(double a) { return __double_as_longlong(a) < 0; }
__device__ __forceinline__ double neg(double a) {
  return __longlong_as_double(__double_as_longlong(a) ^ (long long)0x8000000000000000ull);
}
__device__ __forceinline__ double abs_bits(double a) {
  return __longlong_as_double(__double_as_longlong(a) & 0x7FFFFFFFFFFFFFFFll);
}
__device__ __forceinline__ double max_nn(double a, double b) { return lt_nn(a, b) ? b : a; }

// Select without arithmetic: v if keep, else 0.0 (integer select on the bit pattern).
__device__ __forceinline__ double keep_or_zero(double v, bool keep) {
  long long b = __double_as_longlong(v);
  return __longlong_as_double(keep ? b : 0ll);
}

// --------------------------------------------------------------------------------------------
// Close-encounter predicate over an interval h at critical radius R: minimum distance of the
// straight-line relative motion below R (strict).  Every operation is one IEEE FP64 operation
// in a fixed order without contraction, so every caller on any device decides identically on
// identical inputs.  d = x_b - x_a, dv = v_b - v_a (either order gives the same bits).
// --------------------------------------------------------------------------------------------
__device__ __forceinline__ bool encounter_exact(double dx, double dy, double dz, double dvx,
                                                double dvy, double dvz, double R, double h) {
  const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
  const double v2 = __dadd_rn(__dadd_rn(__dmul_rn(dvx, dvx), __dmul_rn(dvy, dvy)), __dmul_rn(dvz, dvz));
  const double vr = __dadd_rn(__dadd_rn(__dmul_rn(dx, dvx), __dmul_rn(dy, dvy)), __dmul_rn(dz, dvz));
  const double R2 = __dmul_rn(R, R);
  if (r2 < R2) return true;
  if (vr >= 0.0) return false;
  const double t = __ddiv_rn(-vr, v2);
  if (t < h) return __dsub_rn(r2, __ddiv_rn(__dmul_rn(vr, vr), v2)) < R2;
  return __dadd_rn(r2, __dmul_rn(h, __dadd_rn(__dmul_rn(2.0, vr), __dmul_rn(h, v2)))) < R2;
}

// Partition function of order l: the degree-(2l+1) polynomial rising from 0 to 1 on [0, 1]
// with its first l derivatives zero at both ends, f_l(x) = x^{l+1} sum_k C(l+k,k) C(2l+1,l-k)
// (-x)^k, clamped outside [0, 1] (Sec. 3 uses l = 3).
__device__ __forceinline__ double binom_d(int n, int k) {
  double r = 1.0;
  for (int i = 1; i <= k; ++i) r = r * (double)(n - k + i) / (double)i;
  return r;
}

__device__ __forceinline__ double partition_fn(double x, int l) {
  if (__double_as_longlong(x) <= 0ll) return 0.0;             // x <= 0 (or -0)
  if (!lt_nn(x, 1.0)) return 1.0;                             // x >= 1
  if (l == 3) {
    // x^4 (35 - 84 x + 70 x^2 - 20 x^3)
    const double x2 = x * x;
    return x2 * x2 * fma(x, fma(x, fma(x, -20.0, 70.0), -84.0), 35.0);
  }
  double s = 0.0, xk = 1.0;
  for (int k = 0; k <= l; ++k) {
    s += binom_d(l + k, k) * binom_d(2 * l + 1, l - k) * xk;
    xk *= -x;
  }
  double xp = 1.0;
  for (int k = 0; k <= l; ++k) xp *= x;
  return xp * s;
}

// --------------------------------------------------------------------------------------------
// Exact accumulation of doubles: 68 signed 32-bit-digit slots in int64 (carry-save), digit k
// weighing 2^(32k - 1088), plus one slot counting non-finite inputs.  Integer addition is
// associative, so the total is independent of the order of the atomics; sa_round returns it
// correctly rounded to nearest-even.
// --------------------------------------------------------------------------------------------
__device__ __forceinline__ void sa_add(unsigned long long *dig, double x) {
  if (x == 0.0) return;
  const long long bits = __double_as_longlong(x);
  int ex = (int)((bits >> 52) & 0x7FF);
  unsigned long long mant = (unsigned long long)bits & 0xFFFFFFFFFFFFFull;
  if (ex == 0x7FF) { atomicAdd(&dig[SA_NDIG], 1ull); return; }
  if (ex == 0) ex = 1; else mant |= 1ull << 52;
  const int p = ex + 13;  // weight of the mantissa's lowest bit, in units of 2^-1088
  const int k = p >> 5, sh = p & 31;
  const unsigned long long lo = mant << sh;
  const unsigned long long hi = sh ? (mant >> (64 - sh)) : 0ull;
  long long c0 = (long long)(lo & 0xFFFFFFFFull), c1 = (long long)(lo >> 32), c2 = (long long)hi;
  if (bits < 0) { c0 = -c0; c1 = -c1; c2 = -c2; }
  if (c0) atomicAdd(&dig[k], (unsigned long long)c0);
  if (c1) atomicAdd(&dig[k + 1], (unsigned long long)c1);
  if (c2) atomicAdd(&dig[k + 2], (unsigned long long)c2);
}

// Carry propagation in place (one thread): the same value with digits 0..SA_NDIG-2 in [0, 2^32)
// and the sign in the top digit.  A CTA that has summed many terms into its own digits adds them
// to a shared accumulator in this form, so each atomic brings less than 2^32 per digit and the
// shared digits stay far from overflow however many CTAs contribute.
__device__ inline void sa_carry(unsigned long long *dig) {
  for (int k = 0; k < SA_NDIG - 1; ++k) {
    const long long v = (long long)dig[k];
    const long long c = v >> 32;
    dig[k] = (unsigned long long)(v - c * 4294967296ll);
    dig[k + 1] = (unsigned long long)((long long)dig[k + 1] + c);
  }
}

__device__ inline double sa_round(const unsigned long long *in) {
  if (in[SA_NDIG] != 0ull) return __longlong_as_double(0x7FF8000000000000ll);
  long long d[SA_NDIG];
  for (int k = 0; k < SA_NDIG; ++k) d[k] = (long long)in[k];
  for (int k = 0; k < SA_NDIG - 1; ++k) {
    const long long c = d[k] >> 32;
    d[k] -= c * 4294967296ll;
    d[k + 1] += c;
  }
  const bool neg = d[SA_NDIG - 1] < 0;
  if (neg) {
    for (int k = 0; k < SA_NDIG; ++k) d[k] = -d[k];
    for (int k = 0; k < SA_NDIG - 1; ++k) {
      const long long c = d[k] >> 32;
      d[k] -= c * 4294967296ll;
      d[k + 1] += c;
    }
  }
  int t = SA_NDIG - 1;
  while (t >= 0 && d[t] == 0) --t;
  if (t < 0) return 0.0;
  const unsigned long long dt = (unsigned long long)d[t];
  const unsigned long long d1 = t >= 1 ? (unsigned long long)d[t - 1] : 0ull;
  const unsigned long long d2 = t >= 2 ? (unsigned long long)d[t - 2] : 0ull;
  bool sticky = false;
  for (int k = 0; k < t - 2; ++k) sticky |= (d[k] != 0);
  const int lz = __clz((unsigned)dt);
  const unsigned long long H = (dt << 32) | d1;
  unsigned long long T;
  if (lz == 0) {
    T = H;
    sticky |= (d2 != 0ull);
  } else {
    T = (H << lz) | (d2 >> (32 - lz));
    sticky |= ((d2 << lz) & 0xFFFFFFFFull) != 0ull;
  }
  int E = t * 32 + 31 - lz - 1088;  // exponent of the leading bit
  double r;
  if (E < -1022) {
    // below the normal range the exact sum (a multiple of 2^-1074) is representable
    r = 0.0;
    for (int k = t; k >= 0; --k) r += ldexp((double)d[k], 32 * k - 1088);
  } else {
    unsigned long long mant = T >> 11;
    const bool rbit = (T >> 10) & 1ull;
    sticky |= (T & 0x3FFull) != 0ull;
    if (rbit && (sticky || (mant & 1ull))) {
      ++mant;
      if (mant == (1ull << 53)) { mant >>= 1; ++E; }
    }
    if (E > 1023) r = __longlong_as_double(0x7FF0000000000000ll);
    else r = ldexp((double)mant, E - 52);
  }
  return neg ? -r : r;
}

// --------------------------------------------------------------------------------------------
// Kepler drift (Danby 1988, f and g functions): advance (x, v) by dt on the orbit of parameter
// mu.  Elliptic orbits solve for the eccentric-anomaly difference X of
//   X - ec sin X + es (1 - cos X) = n dt,  ec = 1 - r0/a, es = u / (n a^2)
// with Danby's quartically convergent iteration from X = n dt, falling back to a bracketed
// Newton-bisection; other orbits use universal variables with Stumpff functions.
// Returns SYMBA_OK or SYMBA_E_KEPLER / SYMBA_E_NONFINITE.
// --------------------------------------------------------------------------------------------
__device__ inline void stumpff4(double z, double c[4]) {
  if (fabs(z) < 0.1) {
    for (int k = 0; k < 4; ++k) {
      double term = 1.0, s = 0.0;
      for (int i = 2; i <= k; ++i) term /= (double)i;
      for (int j = 0; j < 24; ++j) {
        s += term;
        term *= -z / ((double)(2 * j + k + 1) * (double)(2 * j + k + 2));
      }
      c[k] = s;
    }
    return;
  }
  if (z > 0.0) {
    const double sz = sqrt(z);
    double sn, cs;
    sincos(sz, &sn, &cs);
    c[0] = cs;
    c[1] = sn / sz;
  } else {
    const double sz = sqrt(-z);
    c[0] = cosh(sz);
    c[1] = sinh(sz) / sz;
  }
  c[2] = (1.0 - c[0]) / z;
  c[3] = (1.0 - c[1]) / z;
}

// X - sin X = X^3 (1/3! - X^2/5! + X^4/7! - ...) in Horner form for |X| < 1/2 (through X^19,
// the rest below 1e-21 relative), where the direct difference loses digits to cancellation
__device__ inline double x_minus_sin(double X) {
  if (fabs(X) >= 0.5) return X - sin(X);
  const double z = X * X;
  double p = -1.0 / 121645100408832000.0;                       // -1/19!
  p = fma(p, z, 1.0 / 355687428096000.0);                       // 1/17!
  p = fma(p, z, -1.0 / 1307674368000.0);                        // -1/15!
  p = fma(p, z, 1.0 / 6227020800.0);                            // 1/13!
  p = fma(p, z, -1.0 / 39916800.0);                             // -1/11!
  p = fma(p, z, 1.0 / 362880.0);                                // 1/9!
  p = fma(p, z, -1.0 / 5040.0);                                 // -1/7!
  p = fma(p, z, 1.0 / 120.0);                                   // 1/5!
  p = fma(p, z, -1.0 / 6.0);                                    // -1/3!
  return -(X * z) * p;
}

// The new state is x0 + ((f - 1) x0 + g v0), v0 + (f' x0 + (g' - 1) v0): f - 1 and g' - 1 are
// formed apart from the 1, which they would be rounded into when small.
__device__ inline int kepler_drift(double mu, double dt, double &x, double &y, double &z,
                                   double &vx, double &vy, double &vz) {
  const double r0 = sqrt(fma(z, z, fma(y, y, x * x)));
  const double v2 = fma(vz, vz, fma(vy, vy, vx * vx));
  const double u = fma(z, vz, fma(y, vy, x * vx));
  const double alpha = 2.0 * mu / r0 - v2;
  if (!(r0 > 0.0) || !isfinite(alpha) || !isfinite(u)) return SYMBA_E_NONFINITE;
  double fm1, g, fdot, gdm1;
  if (alpha > 0.0) {
    const double a = mu / alpha;
    const double nn = sqrt(mu / (a * a * a));
    const double ec = 1.0 - r0 / a;
    const double es = u / (nn * a * a);
    const double ndt = nn * dt;
    double X = ndt, sx = 0.0, cx = 1.0;
    bool ok = false;
    for (int it = 0; it < 12; ++it) {
      sincos(X, &sx, &cx);
      const double omc = (cx > 0.0) ? sx * sx / (1.0 + cx) : 1.0 - cx;
      const double F = X - ec * sx + es * omc - ndt;
      const double Fp = 1.0 - ec * cx + es * sx;
      const double Fpp = ec * sx + es * cx;
      const double Fppp = ec * cx - es * sx;
      const double d1 = -F / Fp;
      const double d2 = -F / (Fp + 0.5 * d1 * Fpp);
      const double d3 = -F / (Fp + 0.5 * d2 * Fpp + d2 * d2 * Fppp * (1.0 / 6.0));
      X += d3;
      if (fabs(d3) <= 1e-15 * fmax(1.0, fabs(X))) { ok = true; break; }
    }
    if (!ok) {
      double lo = ndt - 2.5, hi = ndt + 2.5;
      X = ndt;
      for (int it = 0; it < 200; ++it) {
        sincos(X, &sx, &cx);
        const double omc = (cx > 0.0) ? sx * sx / (1.0 + cx) : 1.0 - cx;
        const double F = X - ec * sx + es * omc - ndt;
        const double Fp = 1.0 - ec * cx + es * sx;
        if (F > 0.0) hi = X; else lo = X;
        const double dX = -F / Fp;
        double Xn = X + dX;
        if (fabs(dX) <= 1e-15 * fmax(1.0, fabs(X))) { X = Xn; ok = true; break; }
        if (!(Xn > lo && Xn < hi)) Xn = 0.5 * (lo + hi);
        X = Xn;
      }
      if (!ok) return SYMBA_E_KEPLER;
    }
    sincos(X, &sx, &cx);
    const double omc = (cx > 0.0) ? sx * sx / (1.0 + cx) : 1.0 - cx;
    const double r = a * (1.0 - ec * cx + es * sx);
    fm1 = -(a / r0) * omc;
    g = dt - x_minus_sin(X) / nn;
    fdot = -(a * a * nn * sx) / (r * r0);
    gdm1 = -(a / r) * omc;
  } else {
    const double sgn = dt >= 0.0 ? 1.0 : -1.0;
    double c[4];
    double lo = 0.0, hi = fabs(dt) / r0;
    if (hi == 0.0) return SYMBA_OK;
    bool found = false;
    for (int it = 0; it < 200; ++it) {
      const double s = sgn * hi;
      stumpff4(alpha * s * s, c);
      const double F = r0 * s * c[1] + u * s * s * c[2] + mu * s * s * s * c[3] - dt;
      if (sgn * F >= 0.0) { found = true; break; }
      lo = hi;
      hi *= 2.0;
    }
    if (!found) return SYMBA_E_KEPLER;
    double sa = 0.5 * (lo + hi);
    bool ok = false;
    for (int it = 0; it < 400; ++it) {
      const double s = sgn * sa;
      stumpff4(alpha * s * s, c);
      const double G1 = s * c[1], G2 = s * s * c[2], G3 = s * s * s * c[3];
      const double F = r0 * G1 + u * G2 + mu * G3 - dt;
      const double Fp = r0 * c[0] + u * G1 + mu * G2;
      if (sgn * F > 0.0) hi = sa; else lo = sa;
      const double ds = -F / Fp;
      double sn = sa + sgn * ds;
      if (fabs(ds) <= 1e-15 * fmax(1e-300, fabs(sa))) { sa = sn; ok = true; break; }
      if (!(sn > lo && sn < hi)) sn = 0.5 * (lo + hi);
      sa = sn;
    }
    if (!ok) return SYMBA_E_KEPLER;
    const double s = sgn * sa;
    stumpff4(alpha * s * s, c);
    const double G1 = s * c[1], G2 = s * s * c[2], G3 = s * s * s * c[3];
    const double r = r0 * c[0] + u * G1 + mu * G2;
    fm1 = -mu * G2 / r0;
    g = dt - mu * G3;
    fdot = -mu * G1 / (r * r0);
    gdm1 = -mu * G2 / r;
  }
  const double x0 = x, y0 = y, z0 = z, vx0 = vx, vy0 = vy, vz0 = vz;
  x = x0 + fma(fm1, x0, g * vx0);
  y = y0 + fma(fm1, y0, g * vy0);
  z = z0 + fma(fm1, z0, g * vz0);
  vx = vx0 + fma(gdm1, vx0, fdot * x0);
  vy = vy0 + fma(gdm1, vy0, fdot * y0);
  vz = vz0 + fma(gdm1, vz0, fdot * z0);
  return SYMBA_OK;
}

// --------------------------------------------------------------------------------------------
// Short-interval Kepler drift by the Lagrange f and g series (used on the deep recursion levels,
// where the sub-step h is a tiny fraction of the orbit).  With u = mu/r^3, p = (x.v)/r^2,
// q = v^2/r^2 - u, the derivatives of f and g obey f^(n+1) = (dA_n/dt - u B_n) f + (A_n + dB_n/dt) f'
// with du/dt = -3up, dp/dt = q - 2p^2, dq/dt = -p(u + 2q), which gives, through t^6,
//   f = 1 - u t^2/2 + u p t^3/2 + (3uq - 15up^2 + u^2) t^4/24 + (7up^3 - 3upq - u^2 p) t^5/8
//       + (-945up^4 + 630up^2 q - 45uq^2 + 210u^2p^2 - 24u^2 q - u^3) t^6/720
//   g = t - u t^3/6 + u p t^4/4 + (9uq - 45up^2 + u^2) t^5/120 + (14up^3 - 6upq - u^2 p) t^6/24
// and f', g' by term-wise differentiation.  Used only when x = t max(sqrt u, |p|, sqrt|q|)
// <= 2e-3, so the first omitted terms are below 1e-17 relative; for x < 3.2e-5 the series stops
// after t^3 and for x < 1e-6 after t^2 (the omitted terms are then below 1.1e-18).  The order is
// chosen from an FP32 estimate of s = x^2 with a factor-2 margin on each threshold.  Returns false
// (state untouched) when the interval is too long for the series.
// --------------------------------------------------------------------------------------------
__device__ __forceinline__ float f32_trunc(double a) {
  // FP64 -> FP32 by bit manipulation (truncation; no FP64-pipe conversion); for |a| in the normal
  // FP32 range, relative error < 2^-23, which the order decision below leaves margin for
  // (|a| bits << 3 | the next 3 mantissa bits) carries the exponent's low 9 bits over the FP32
  // exponent field; adding 2^30 re-biases it (1023 - 127 = 896 = 512 + 384) for every exponent
  // of the normal FP32 range.  Below it: +0; above it (and Inf, NaN): Inf with the sign.
  const unsigned hi = (unsigned)__double2hiint(a), lo = (unsigned)__double2loint(a);
  const unsigned mag = hi & 0x7FFFFFFFu;
  unsigned r = __funnelshift_l(lo, mag, 3) + 0x40000000u;
  r = mag >= 0x47F00000u ? 0x7F800000u : r;
  r |= hi & 0x80000000u;
  return __uint_as_float(mag < 0x38100000u ? 0u : r);
}

__device__ __forceinline__ bool drift_series(double mu, double t, double &x, double &y, double &z,
                                             double &vx, double &vy, double &vz) {
  // order decision in FP32 (2x margin on every threshold): s = x^2 bounds the first term
  const float xf = f32_trunc(x), yf = f32_trunc(y), zf = f32_trunc(z);
  const float vxf = f32_trunc(vx), vyf = f32_trunc(vy), vzf = f32_trunc(vz);
  const float r2f = fmaf(zf, zf, fmaf(yf, yf, xf * xf));
  const float rif = rsqrtf(r2f), ri2f = rif * rif;
  const float uf = f32_trunc(mu) * ri2f * rif;
  const float pf = fmaf(zf, vzf, fmaf(yf, vyf, xf * vxf)) * ri2f;
  const float qf = fmaf(fmaf(vzf, vzf, fmaf(vyf, vyf, vxf * vxf)), ri2f, -uf);
  const float tf = f32_trunc(t);
  const float sf = fmaxf(fmaxf(uf, pf * pf), fabsf(qf)) * tf * tf;
  if (!(sf <= 2.0e-6f)) return false;
  const double r2 = fma(z, z, fma(y, y, x * x));
  const double ri = rsqrt_fp64(r2);
  const double ri2 = ri * ri;
  const double u = mu * ri2 * ri;
  const double t2 = t * t;
  const double x0 = x, y0 = y, z0 = z;
  // In v' the term f' x is already ~x of v (x = n t), so f' needs one order more than f, g and
  // g': (3/2) u p t^2 at order 2 (up to 1.5 x^2 of v, 7e-13) and (3uq - 15up^2 + u^2) t^3/6 at
  // order 3 (up to 3.3e-14 of v).  Their size lets FP32 (the decision's u, p, q) supply them.
  if (sf < 5e-13f) {
    // x < 1e-6: f - 1, g, g' - 1 to order t^2, f' = -u t (1 - 3/2 p t) to t^2; the rest of the
    // series moves x' and v' by a few 1e-18 at most
    const double fm1 = t2 * (-0.5 * u), fd0 = -u * t;
    const double fd = fma(fd0, (double)(-1.5f * pf * tf), fd0);
    x = fma(fm1, x0, fma(t, vx, x0));
    y = fma(fm1, y0, fma(t, vy, y0));
    z = fma(fm1, z0, fma(t, vz, z0));
    vx = fma(fd, x0, fma(fm1, vx, vx));
    vy = fma(fd, y0, fma(fm1, vy, vy));
    vz = fma(fd, z0, fma(fm1, vz, vz));
    return true;
  }
  const double p = fma(z, vz, fma(y, vy, x * vx)) * ri2;
  double fm1, gmt, fd, gdm1;
  if (sf < 5e-10f) {
    // x < 3.2e-5: f - 1, g, g' - 1 to order t^3, f' to t^3 (its t^3 term, (3uq - 15up^2 + u^2)
    // t^3/6, in FP32); the rest of the series moves x' and v' by a few 1e-18 at most
    const double up = u * p;
    fm1 = t2 * fma(t, 0.5 * up, -0.5 * u);
    gmt = t2 * t * (-u * (1.0 / 6.0));
    fd = t * fma(t, 1.5 * up, -u) +
         (double)((3.0f * uf * qf - 15.0f * uf * pf * pf + uf * uf) * (1.0f / 6.0f) * tf * tf * tf);
    gdm1 = t2 * fma(t, up, -0.5 * u);
  } else {
    const double v2 = fma(vz, vz, fma(vy, vy, vx * vx));
    const double q = fma(v2, ri2, -u);
    const double up = u * p, uq = u * q, u2 = u * u, p2 = p * p;
    const double c4 = (3.0 * uq - 15.0 * up * p + u2) * (1.0 / 24.0);
    const double c5 = (7.0 * up * p2 - 3.0 * up * q - u2 * p) * 0.125;
    const double c6 = (-945.0 * up * p2 * p + 630.0 * up * p * q - 45.0 * uq * q + 210.0 * u2 * p2
                       - 24.0 * u2 * q - u2 * u) * (1.0 / 720.0);
    const double d5 = (9.0 * uq - 45.0 * up * p + u2) * (1.0 / 120.0);
    const double d6 = (14.0 * up * p2 - 6.0 * up * q - u2 * p) * (1.0 / 24.0);
    fm1 = t2 * fma(t, fma(t, fma(t, fma(t, c6, c5), c4), 0.5 * up), -0.5 * u);
    gmt = t2 * t * fma(t, fma(t, fma(t, d6, d5), 0.25 * up), -u * (1.0 / 6.0));
    fd = t * fma(t, fma(t, fma(t, fma(t, 6.0 * c6, 5.0 * c5), 4.0 * c4), 1.5 * up), -u);
    gdm1 = t2 * fma(t, fma(t, fma(t, 6.0 * d6, 5.0 * d5), up), -0.5 * u);
  }
  x = fma(fm1, x0, fma(gmt, vx, fma(t, vx, x0)));
  y = fma(fm1, y0, fma(gmt, vy, fma(t, vy, y0)));
  z = fma(fm1, z0, fma(gmt, vz, fma(t, vz, z0)));
  vx = fma(fd, x0, fma(gdm1, vx, vx));
  vy = fma(fd, y0, fma(gdm1, vy, vy));
  vz = fma(fd, z0, fma(gdm1, vz, vz));
  return true;
}

// --------------------------------------------------------------------------------------------
// host-side launch wrappers (defined in the kernel translation units)
// --------------------------------------------------------------------------------------------
struct LaunchCfg {
  int sms;            // multiprocessors
  int trap_blocks;    // persistent trapezoid grid
  int rec_blocks;     // persistent recursion grid
};

void launch_setup_disk(const Dev &D, int d, cudaStream_t s);
void launch_init_state(const Dev &D, int d, int n, const double *xh, const double *vh,
                       const double *m, const double *rad, const double *rh, int compute_rh,
                       cudaStream_t s);
void launch_momentum(const Dev &D, int ndisks, cudaStream_t s);
void launch_sundrift(const Dev &D, long long npart, int pre, cudaStream_t s);
void launch_trap(const Dev &D, const LaunchCfg &L, int mode, int precision, cudaStream_t s);
void launch_reduce(const Dev &D, long long npart, int precision, cudaStream_t s);
void launch_split(const Dev &D, long long npart, cudaStream_t s);
void launch_groups(const Dev &D, int ndisks, cudaStream_t s);
void launch_drift(const Dev &D, long long npart, cudaStream_t s);
void launch_recursion(const Dev &D, const LaunchCfg &L, cudaStream_t s);
void launch_energy(const Dev &D, int d, const LaunchCfg &L, unsigned long long *acc /*4*(SA_NDIG+1)*/,
                   cudaStream_t s);
void launch_energy_round(unsigned long long *acc, double *out4, cudaStream_t s);
void launch_gather_state(const Dev &D, int d, int n, double *x, double *v, double *m, double *rad,
                         int *alive, double *rh, cudaStream_t s);
void launch_scatter_state(const Dev &D, int d, int n, const double *x, const double *v,
                          cudaStream_t s);
void launch_prologue(const Dev &D, int ndisks, cudaStream_t s);
void launch_field(const Dev &D, int mode, int precision, cudaStream_t s);
void launch_discard(const Dev &D, long long npart, cudaStream_t s);
int trap_blocks_per_sm(int precision);
int recursion_blocks_per_sm();
bool order_groups_init();
void launch_order_groups(const Dev &D, cudaStream_t s);
void launch_state_hash(const Dev &D, long long np, int ndisks, unsigned long long *h, cudaStream_t s);
