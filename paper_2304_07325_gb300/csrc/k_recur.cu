// Recursive sub-stepping of the encounter groups (Sec. 2: groups integrated in parallel, the pairs
// of a group sequentially; Sec. 3: subdivision factor M, shell ratio R_k/R_{k+1}, partition
// function f_l).  One warp integrates one group through M x E_1(tau / M), where
//   E_k(h): (i)   check the pairs of F_{k-1} at shell k over h -> F_k (a pair whose current
//                 separation is below R_i + R_j merges instead);
//           (ii)  kick h/2 with the level-k share w_k = g_k - g_{k-1} of every F_{k-1} force;
//           (iii) bodies of F_{k-1} in no F_k pair drift h; the rest run M x E_{k+1}(h/M);
//           (iv)  kick h/2 as in (ii).
// The recursion is a loop over an explicit level stack.  Every pair carries a level mark lev
// (the deepest k with the pair in F_k on the current path), so F_k = {lev >= k}; running E_{k+1}
// on all components of F_k at once equals running it per component because components share no
// body.  The active pairs F_{k-1} and their bodies are kept as nested prefixes of two
// permutations (stable partition after every check), so deep levels touch only their own pairs.
//
// The sub-step chain is latency-bound (GB300 issues one FP64 instruction per ~64 cycles per warp),
// so it is kept short:
//   - the group's bodies and pairs are gathered into a member-slot view that lives in shared
//     memory for groups of up to 32 bodies and 64 pairs (global scratch otherwise), so phases
//     exchange data through shared memory, and are scattered back at the end;
//   - the deep-level drift uses the Lagrange f and g series when the sub-step is a tiny fraction
//     of the orbit; square roots come from an integer-built FP32 seed plus one FP64 correction;
//     the shell weights use per-level reciprocal tables;
//   - the forces of the closing kick of one sub-step are reused by the opening kick of the next
//     (same positions, same pairs, same weights);
//   - once F_{k-1} holds a single pair -- the close or bound pairs whose chains set the step
//     time -- the sub-steps of levels >= k run in the single-pair path (pair_run), the two
//     bodies packed component-wise across the warp (details at pair_run).
// Groups of at most 32 bodies and 32 pairs keep their state in registers (run_group_regs).
// The check below level 0 uses the division-free form of the predicate (same minimum-distance
// test; identical except at exact ties).
#include "internal.cuh"

#define FULL 0xffffffffu
#define SMALL_M 32
#define SMALL_P 64

// member-slot-indexed state of one group
struct GView {
  double *x, *y, *z, *vx, *vy, *vz, *m, *gm, *rad, *rh;
  int *alive;
  int *pa, *pb, *lev;          // pair -> member slots, level mark
  double *R0, *invR0, *pf;     // critical radius, its inverse, forces [pair][5]
  int *adj_off, *adj_cnt, *adj;
  int *perm, *ptmp, *mperm, *mtmp;
};

struct SmallView {             // shared-memory backing of a small group
  double x[SMALL_M], y[SMALL_M], z[SMALL_M], vx[SMALL_M], vy[SMALL_M], vz[SMALL_M];
  double m[SMALL_M], gm[SMALL_M], rad[SMALL_M], rh[SMALL_M];
  double R0[SMALL_P], invR0[SMALL_P], pf[5 * SMALL_P];
  int alive[SMALL_M], adj_off[SMALL_M], adj_cnt[SMALL_M], mperm[SMALL_M], mtmp[SMALL_M];
  int pa[SMALL_P], pb[SMALL_P], lev[SMALL_P], perm[SMALL_P], ptmp[SMALL_P], adj[2 * SMALL_P];
};

struct GroupCtx {
  int d, moff, mcnt, poff, pcnt;
  int M, l, max_depth, max_substeps;
  double dt, lam, G, mu, invM;
  const DiskDesc *dp;
};

// h / M; for M a power of two the product with 1/M is the same number without a division
__device__ __forceinline__ double sub_interval(const GroupCtx &C, double h) {
  return (C.M & (C.M - 1)) == 0 ? h * C.invM : h / (double)C.M;
}

__device__ __forceinline__ bool contact(const GView &S, int a, int b) {
  const double dx = __dsub_rn(S.x[b], S.x[a]), dy = __dsub_rn(S.y[b], S.y[a]), dz = __dsub_rn(S.z[b], S.z[a]);
  const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
  const double Rc = __dadd_rn(S.rad[a], S.rad[b]);
  return r2 < __dmul_rn(Rc, Rc);
}

// minimum distance of the straight-line relative motion over [0, h] below R_k (division-free;
// comparisons of non-negative values on their bit patterns)
__device__ __forceinline__ bool predicate_fast(const GView &S, int a, int b, double R2, double h) {
  const double dx = S.x[b] - S.x[a], dy = S.y[b] - S.y[a], dz = S.z[b] - S.z[a];
  const double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
  if (lt_nn(r2, R2)) return true;
  const double dvx = S.vx[b] - S.vx[a], dvy = S.vy[b] - S.vy[a], dvz = S.vz[b] - S.vz[a];
  const double vr = fma(dz, dvz, fma(dy, dvy, dx * dvx));
  if (!is_neg(vr)) return false;
  const double v2 = fma(dvz, dvz, fma(dvy, dvy, dvx * dvx));
  const double hv2 = h * v2;
  if (lt_nn(neg(vr), hv2)) return lt_nn(fma(r2, v2, -vr * vr), R2 * v2);
  const double e = fma(h, fma(h, v2, 2.0 * vr), r2);
  return is_neg(e) || lt_nn(e, R2);
}

// squared separation (FMA form) and whether the exact contact test is needed at all: contact
// requires r2 < (R_a + R_b)^2, and the FMA-form r2 is within a few ulp of the exact one
__device__ __forceinline__ bool near_contact(const GView &S, int a, int b) {
  const double dx = S.x[b] - S.x[a], dy = S.y[b] - S.y[a], dz = S.z[b] - S.z[a];
  const double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
  const double Rc = S.rad[a] + S.rad[b];
  return lt_nn(r2, 1.0000001 * (Rc * Rc));
}

__device__ __forceinline__ void set_r0(const GView &S, const GroupCtx &C, int q) {
  const double R0 = __dmul_rn(C.lam, __dadd_rn(S.rh[S.pa[q]], S.rh[S.pb[q]]));
  S.R0[q] = R0;
  S.invR0[q] = R0 > 0.0 ? 1.0 / R0 : 0.0;
}

// merger of b into a (a holds the lower index): summed mass, mass-weighted position and
// barycentric velocity, radius (R_a^3 + R_b^3)^{1/3}, Hill radius rH_a (m / m_a)^{1/3}; b leaves
// the system.
__device__ void merge_pair(const GView &S, const GroupCtx &C, const Dev &D, int a, int b) {
  const double ma = S.m[a], mb = S.m[b];
  const double M = __dadd_rn(ma, mb);
  if (M > 0.0) {
    S.x[a] = __ddiv_rn(__dadd_rn(__dmul_rn(ma, S.x[a]), __dmul_rn(mb, S.x[b])), M);
    S.y[a] = __ddiv_rn(__dadd_rn(__dmul_rn(ma, S.y[a]), __dmul_rn(mb, S.y[b])), M);
    S.z[a] = __ddiv_rn(__dadd_rn(__dmul_rn(ma, S.z[a]), __dmul_rn(mb, S.z[b])), M);
    S.vx[a] = __ddiv_rn(__dadd_rn(__dmul_rn(ma, S.vx[a]), __dmul_rn(mb, S.vx[b])), M);
    S.vy[a] = __ddiv_rn(__dadd_rn(__dmul_rn(ma, S.vy[a]), __dmul_rn(mb, S.vy[b])), M);
    S.vz[a] = __ddiv_rn(__dadd_rn(__dmul_rn(ma, S.vz[a]), __dmul_rn(mb, S.vz[b])), M);
  }
  const double Ra = S.rad[a], Rb = S.rad[b];
  S.rad[a] = cbrt_rn(__dadd_rn(__dmul_rn(__dmul_rn(Ra, Ra), Ra), __dmul_rn(__dmul_rn(Rb, Rb), Rb)));
  if (ma > 0.0) S.rh[a] = __dmul_rn(S.rh[a], cbrt_rn(__ddiv_rn(M, ma)));
  S.m[a] = M;
  S.gm[a] = __dmul_rn(C.G, M);
  S.m[b] = 0.0;
  S.gm[b] = 0.0;
  S.rad[b] = 0.0;
  S.rh[b] = 0.0;
  S.alive[b] = 0;
  atomicAdd(&D.stat[C.d].merges, 1ull);
  const int ao = S.adj_off[a], ac = S.adj_cnt[a];
  for (int e = 0; e < ac; ++e) set_r0(S, C, S.adj[ao + e] >> 1);
}

// stable partition of idx[0..len): entries with pred true first; returns their count
template <class Pred>
__device__ int partition_prefix(int *idx, int *tmp, int len, Pred pred, int lane) {
  int ntrue = 0;
  for (int b = 0; b < len; b += 32) {
    const int i = b + lane;
    const bool f = i < len && pred(idx[i]);
    ntrue += __popc(__ballot_sync(FULL, f));
  }
  int ct = 0, cf = ntrue;
  const unsigned below = (1u << lane) - 1u;
  for (int b = 0; b < len; b += 32) {
    const int i = b + lane;
    const bool in = i < len;
    const int v = in ? idx[i] : 0;
    const bool f = in && pred(v);
    const unsigned bt = __ballot_sync(FULL, f), bf = __ballot_sync(FULL, in && !f);
    if (f) tmp[ct + __popc(bt & below)] = v;
    else if (in) tmp[cf + __popc(bf & below)] = v;
    ct += __popc(bt);
    cf += __popc(bf);
  }
  __syncwarp();
  for (int i = lane; i < len; i += 32) idx[i] = tmp[i];
  __syncwarp();
  return ntrue;
}

struct Levels {
  double *h;
  int *cnt, *lenL, *lenM;
};

// (i): level-k check of F_{k-1} (the first lenL[k] entries of perm).  Returns whether F_k is
// non-empty; sets *merged when bodies merged.
__device__ bool check_level(const GView &S, const GroupCtx &C, const Dev &D, const Levels &V, int k,
                            int lane, bool *merged) {
  const int L = V.lenL[k];
  const double h = V.h[k];
  bool any_contact = false;
  for (int b = 0; b < L; b += 32) {
    const int t = b + lane;
    bool ct = false;
    if (t < L) {
      const int q = S.perm[t];
      const int a = S.pa[q], c = S.pb[q];
      if (S.alive[a] && S.alive[c] && near_contact(S, a, c)) ct = contact(S, a, c);
    }
    any_contact |= (__any_sync(FULL, ct) != 0);
  }
  const double ck2 = C.dp->ck2[k];
  bool nonempty = false;
  if (!any_contact) {
    for (int b = 0; b < L; b += 32) {
      const int t = b + lane;
      bool fl = false;
      if (t < L) {
        const int q = S.perm[t];
        const int a = S.pa[q], c = S.pb[q];
        if (S.alive[a] && S.alive[c]) {
          const double R0 = S.R0[q];
          fl = predicate_fast(S, a, c, R0 * R0 * ck2, h);
        }
        S.lev[q] = fl ? k : k - 1;
      }
      nonempty |= (__any_sync(FULL, fl) != 0);
    }
    *merged = false;
  } else {
    // a merger changes bodies that later pairs read: take the pairs one by one in list order
    __syncwarp();
    if (lane == 0) {
      for (int q = 0; q < C.pcnt; ++q) {
        if (S.lev[q] < k - 1) continue;
        const int a = S.pa[q], c = S.pb[q];
        bool fl = false;
        if (S.alive[a] && S.alive[c]) {
          if (contact(S, a, c)) merge_pair(S, C, D, a, c);
          else {
            const double R0 = S.R0[q];
            fl = predicate_fast(S, a, c, R0 * R0 * ck2, h);
          }
        }
        S.lev[q] = fl ? k : k - 1;
        nonempty |= fl;
      }
    }
    nonempty = __shfl_sync(FULL, nonempty ? 1 : 0, 0) != 0;
    *merged = true;
  }
  __syncwarp();
  return nonempty;
}

// forces of the level-k share of every F_{k-1} pair at the current positions
__device__ void forces_level(const GView &S, const GroupCtx &C, const Levels &V, int k, int lane) {
  const int L = V.lenL[k];
  const double ck = C.dp->ck[k], ck1 = C.dp->ck[k + 1], idk = C.dp->invdc[k];
  const double idkm = k > 0 ? C.dp->invdc[k - 1] : 0.0;
  for (int t = lane; t < L; t += 32) {
    const int q = S.perm[t];
    const int a = S.pa[q], c = S.pb[q];
    double fi = 0.0, fj = 0.0, dx = 0.0, dy = 0.0, dz = 0.0;
    if (S.alive[a] && S.alive[c]) {
      dx = S.x[c] - S.x[a];
      dy = S.y[c] - S.y[a];
      dz = S.z[c] - S.z[a];
      const double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
      const double ri = rsqrt_fp64(r2);
      const double rho = r2 * ri * S.invR0[q];     // r / R_0
      // w_k = g_k - g_{k-1}: the transition zones of g_k and g_{k-1} do not overlap, so at most
      // one of the two is strictly between 0 and 1 -- evaluate only that polynomial
      double w;
      if (k == 0) {
        w = partition_fn((rho - ck1) * idk, C.l);
      } else if (lt_nn(rho, ck)) {                  // r < R_k: g_{k-1} = 0
        w = partition_fn((rho - ck1) * idk, C.l);
      } else {                                      // r >= R_k: g_k = 1
        w = 1.0 - partition_fn((rho - ck) * idkm, C.l);
      }
      const double s = w * (ri * ri * ri);
      fi = S.gm[c] * s;
      fj = S.gm[a] * s;
    }
    double *f = S.pf + 5 * q;
    f[0] = dx; f[1] = dy; f[2] = dz; f[3] = fi; f[4] = fj;
  }
  __syncwarp();
}

// kick hh of the bodies of F_{k-1} (the first lenM[k] member slots of mperm)
__device__ void kick_level(const GView &S, const Levels &V, int k, double hh, int lane) {
  const int L = V.lenM[k];
  for (int t = lane; t < L; t += 32) {
    const int a = S.mperm[t];
    if (!S.alive[a]) continue;
    const int ao = S.adj_off[a], ac = S.adj_cnt[a];
    double ax = 0.0, ay = 0.0, az = 0.0;
    for (int e = 0; e < ac; ++e) {
      const int code = S.adj[ao + e];
      const int q = code >> 1;
      if (S.lev[q] < k - 1) continue;
      const double *f = S.pf + 5 * q;
      if ((code & 1) == 0) { ax = fma(f[3], f[0], ax); ay = fma(f[3], f[1], ay); az = fma(f[3], f[2], az); }
      else { ax = fma(-f[4], f[0], ax); ay = fma(-f[4], f[1], ay); az = fma(-f[4], f[2], az); }
    }
    S.vx[a] = fma(hh, ax, S.vx[a]);
    S.vy[a] = fma(hh, ay, S.vy[a]);
    S.vz[a] = fma(hh, az, S.vz[a]);
  }
  __syncwarp();
}

// (iii): drift h the bodies of mperm[from..to)
__device__ void drift_range(const GView &S, const GroupCtx &C, const Dev &D, int from, int to, double h,
                            int lane) {
  for (int t = from + lane; t < to; t += 32) {
    const int a = S.mperm[t];
    if (!S.alive[a]) continue;
    double x = S.x[a], y = S.y[a], z = S.z[a], vx = S.vx[a], vy = S.vy[a], vz = S.vz[a];
    if (!drift_series(C.mu, h, x, y, z, vx, vy, vz)) {
      const int st = kepler_drift(C.mu, h, x, y, z, vx, vy, vz);
      if (st != SYMBA_OK) set_status(&D.stat[C.d], st);
    }
    S.x[a] = x; S.y[a] = y; S.z[a] = z;
    S.vx[a] = vx; S.vy[a] = vy; S.vz[a] = vz;
  }
  __syncwarp();
}

__device__ __noinline__ int pair_run(const Dev &D, const GroupCtx &C, int lane, double *hs, int *cs,
                                     double *lc, double &Xio, double &Vio, double gA, double gB,
                                     double pR0sq, double piR0, double pRcut, int &kio, int &plev_io,
                                     long long &substeps_io, int &deepest_io);

__device__ void recurse(const GView &S, const GroupCtx &C, const Dev &D, const Levels &V, int lane, double *lc) {
  int k = 1, deepest = 1, forces_at = -1;
  long long substeps = 0;
  V.h[1] = C.dt / (double)C.M;
  V.cnt[1] = 0;
  V.lenL[1] = C.pcnt;
  V.lenM[1] = C.mcnt;
  bool start = true, aborted = false;
  for (;;) {
    if (start) {
      // a single pair below this level: the packed single-pair path
      if (k >= 1 && C.l == 3 && V.lenL[k] == 1) {
        const int q = S.perm[0];
        const int a = S.pa[q], b = S.pb[q];
        if (S.alive[a] && S.alive[b]) {
          const int pc = lane & 3, src = ((lane >> 2) & 1) ? b : a;
          double X = pc == 0 ? S.x[src] : (pc == 1 ? S.y[src] : (pc == 2 ? S.z[src] : 0.0));
          double Vv = pc == 0 ? S.vx[src] : (pc == 1 ? S.vy[src] : (pc == 2 ? S.vz[src] : 0.0));
          const double R0 = S.R0[q], Rc = S.rad[a] + S.rad[b];
          int plev = S.lev[q];
          const int k0 = k;
          __syncwarp();
          const long long sub0 = substeps;
          const int rc = pair_run(D, C, lane, V.h, V.cnt, lc, X, Vv, S.gm[a], S.gm[b], R0 * R0,
                                  S.invR0[q], 1.0000001 * (Rc * Rc), k, plev, substeps, deepest);
          if (lane == 0) atomicAdd(&D.stat[C.d].pair_substeps, (unsigned long long)(substeps - sub0));
          if (lane < 8 && pc < 3) {
            double *px = pc == 0 ? S.x : (pc == 1 ? S.y : S.z);
            double *pv = pc == 0 ? S.vx : (pc == 1 ? S.vy : S.vz);
            px[src] = X;
            pv[src] = Vv;
          }
          if (lane == 0) S.lev[q] = plev;
          // levels entered below k0 hold the same single pair and its two bodies
          for (int i = k0 + 1 + lane; i <= k; i += 32) { V.lenL[i] = 1; V.lenM[i] = V.lenM[k0]; }
          __syncwarp();
          forces_at = -1;
          if (rc == 0) {
            if (k == 0) break;
            start = false;
            continue;
          }
          if (rc == 2) { aborted = true; break; }
        }
      }
      ++substeps;
      if (substeps > C.max_substeps) { aborted = true; break; }
      deepest = max(deepest, k);
      bool merged = false;
      const bool fk = check_level(S, C, D, V, k, lane, &merged);
      if (merged || forces_at != k) { forces_level(S, C, V, k, lane); forces_at = k; }
      kick_level(S, V, k, 0.5 * V.h[k], lane);
      const bool deeper = fk && (k + 1 <= C.max_depth);
      if (fk && !deeper && lane == 0) set_status(&D.stat[C.d], SYMBA_E_DEPTH);
      int lm1 = 0;
      if (deeper) {
        // F_k and its bodies become the prefixes of the next level
        const int lp = partition_prefix(S.perm, S.ptmp, V.lenL[k], [&](int q) { return S.lev[q] == k; }, lane);
        lm1 = partition_prefix(S.mperm, S.mtmp, V.lenM[k],
                               [&](int a) {
                                 const int ao = S.adj_off[a], ac = S.adj_cnt[a];
                                 for (int e = 0; e < ac; ++e)
                                   if (S.lev[S.adj[ao + e] >> 1] >= k) return true;
                                 return false;
                               }, lane);
        V.lenL[k + 1] = lp;
        V.lenM[k + 1] = lm1;
      }
      drift_range(S, C, D, lm1, V.lenM[k], V.h[k], lane);
      if (deeper) {
        ++k;
        V.h[k] = sub_interval(C, V.h[k - 1]);
        V.cnt[k] = 0;
        continue;
      }
      start = false;
    }
    // (iv) of E_k, then the next of its M calls or back to the parent's (iv)
    forces_level(S, C, V, k, lane);
    forces_at = k;
    kick_level(S, V, k, 0.5 * V.h[k], lane);
    if (++V.cnt[k] < C.M) { start = true; continue; }
    --k;
    forces_at = -1;
    if (k == 0) break;
  }
  if (aborted && lane == 0) set_status(&D.stat[C.d], SYMBA_E_DEPTH);
  if (lane == 0) {
    atomicMax(&D.stat[C.d].max_depth, deepest);
    atomicAdd(&D.stat[C.d].substeps, (unsigned long long)substeps);
    atomicMax(&D.stat[C.d].max_chain, (unsigned long long)substeps);
  }
}

// --------------------------------------------------------------------------------------------
// Register-resident path for groups of at most 32 bodies and 32 pairs: lane a holds body a, lane
// q holds pair q (member slots, critical radius, level mark, the last forces).  Pairs read their
// bodies with warp shuffles; F_{k-1} and F_k are ballot masks, a body's pairs a bitmask, so no
// list is stored or partitioned.  Same method, same order of accumulation (pair-list order).
// --------------------------------------------------------------------------------------------
#define SH(v, src) __shfl_sync(FULL, (v), (src))

__device__ __forceinline__ bool contact_regs(double xa, double ya, double za, double xb, double yb,
                                             double zb, double ra, double rb) {
  const double dx = __dsub_rn(xb, xa), dy = __dsub_rn(yb, ya), dz = __dsub_rn(zb, za);
  const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
  const double Rc = __dadd_rn(ra, rb);
  return r2 < __dmul_rn(Rc, Rc);
}

__device__ __forceinline__ bool predicate_regs(double dx, double dy, double dz, double r2, double dvx,
                                               double dvy, double dvz, double R2, double h) {
  if (lt_nn(r2, R2)) return true;
  const double vr = fma(dz, dvz, fma(dy, dvy, dx * dvx));
  if (!is_neg(vr)) return false;
  const double v2 = fma(dvz, dvz, fma(dvy, dvy, dvx * dvx));
  if (lt_nn(neg(vr), h * v2)) return lt_nn(fma(r2, v2, -vr * vr), R2 * v2);
  const double e = fma(h, fma(h, v2, 2.0 * vr), r2);
  return is_neg(e) || lt_nn(e, R2);
}

// --------------------------------------------------------------------------------------------
// One pair alone below level k (F_{k-1} = {q}): every sub-step of levels >= k then touches only
// the pair's two bodies, and a group spends most of its sub-steps there when it holds a close or
// bound pair.  The sub-step chain is latency-bound: GB300 runs one FP64 warp instruction per ~64
// cycles whatever the number of active lanes, and an FP64 result that passes through another
// unit (shuffle, select, integer compare) before the next FP64 instruction costs ~46 cycles more.
// So the warp holds the two bodies component-wise -- lane = 8 cp + 4 b + c: copy cp (0..3) of
// body b (0, 1), component c (x, y, z, and a zero pad) -- which makes
//   - a vector update one FP64 instruction for all components of both bodies;
//   - a sum over components one gather (three shuffles) and two additions, in the order
//     (x + y) + z;
//   - three or four independent operations of a scalar chain one fused multiply-add, copy cp
//     taking the cp-th operands (branch-free bit selects), the results exchanged by shuffles.
// Levels whose shell weight vanishes for the current separation (outside [R_{j+1}, R_{j-1}))
// skip the force and the kick.  The method is the general path's, step by step; the arithmetic
// differs only in rounding (component sums, the weight argument r A + B with per-level
// constants, Estrin's form of f_3, the series coefficients).
// --------------------------------------------------------------------------------------------
__device__ __forceinline__ double fma_rn(double a, double b, double c) {
  double r;
  asm("fma.rn.f64 %0, %1, %2, %3;" : "=d"(r) : "d"(a), "d"(b), "d"(c));
  return r;
}
// a where the mask is set, b elsewhere (one bit-select per 32-bit half, no branch)
__device__ __forceinline__ double bsel(double a, double b, unsigned m) {
  const long long ia = __double_as_longlong(a), ib = __double_as_longlong(b);
  const unsigned lo = ((unsigned)ia & m) | ((unsigned)ib & ~m);
  const unsigned hi = ((unsigned)(ia >> 32) & m) | ((unsigned)(ib >> 32) & ~m);
  return __longlong_as_double((long long)(((unsigned long long)hi << 32) | lo));
}
// four independent fused multiply-adds in one instruction: copy cp evaluates a_cp b_cp + c_cp
// (m0, m1: the bits of cp as masks; a product is a fused multiply-add with -0, which returns it
// exactly, signed zeros included)
__device__ __forceinline__ double fma4(unsigned m0, unsigned m1, double a0, double b0, double c0,
                                       double a1, double b1, double c1, double a2, double b2,
                                       double c2, double a3, double b3, double c3) {
  const double a = bsel(bsel(a3, a2, m0), bsel(a1, a0, m0), m1);
  const double b = bsel(bsel(b3, b2, m0), bsel(b1, b0, m0), m1);
  const double c = bsel(bsel(c3, c2, m0), bsel(c1, c0, m0), m1);
  return fma_rn(a, b, c);
}
// the value copy k holds for this lane's body and component
__device__ __forceinline__ double cpy(double v, int lane, int k) {
  return __shfl_sync(FULL, v, (lane & 7) | (k << 3));
}
// (p_x + p_y) + p_z over the component lanes of this lane's body (base: its x lane)
__device__ __forceinline__ double csum3(double p, int base) {
  const double a = __shfl_sync(FULL, p, base), b = __shfl_sync(FULL, p, base + 1);
  const double c = __shfl_sync(FULL, p, base + 2);
  return (a + b) + c;
}
// The FP32 seed alone: y0f ~ 1/sqrt(r2e), ok when r2e is a normal FP32 number.
__device__ __forceinline__ void seed_f32(float r2e, bool &ok, float &y0f) {
  const unsigned yb = __float_as_uint(r2e);
  const int fe = (int)((yb >> 23) & 0xFF);
  ok = fe >= 1 && fe <= 253 && (int)yb > 0;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y0f) : "f"(ok ? r2e : 1.0f));
}
// y0 = y0f exactly as a double and its exact square t, built on the integer pipe.
__device__ __forceinline__ void seed_expand(float y0f, double &y0, double &t) {
  const unsigned b = __float_as_uint(y0f);
  const int ey = (int)((b >> 23) & 0xFF);
  y0 = __hiloint2double(((ey + 896) << 20) | (int)((b & 0x7FFFFF) >> 3), (int)((b & 7u) << 29));
  const unsigned long long my = (unsigned long long)((b & 0x7FFFFFu) | 0x800000u);
  const unsigned long long p = my * my;
  const int top = (int)(p >> 47);
  const unsigned long long mant = (p << (6 - top)) & 0xFFFFFFFFFFFFFull;
  const long long e2 = 2 * (ey - 127) + top + 1023;
  t = __longlong_as_double((long long)(((unsigned long long)e2 << 52) | mant));
}
// The same seed from an FP32 estimate r2e of r2 (relative error ~2^-22), available before the
// FP64 sum that forms r2: the seed's square t stays exact, so the third-order corrections from
// e = 1 - r2 t still reach full FP64 accuracy.  ok = false when r2e is not a normal FP32 number.
__device__ __forceinline__ void seed_nb(float r2e, double &y0, double &t, bool &ok, float &y0f) {
  seed_f32(r2e, ok, y0f);
  seed_expand(y0f, y0, t);
}
// The double equal to a normal FP32 value, built on the integer pipe (a conversion instruction
// takes the FP64 pipe's rate); FP32 zeros and subnormals give zero.
__device__ __forceinline__ double f32_to_f64(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned e = (b >> 23) & 0xFFu;
  const unsigned hi = (b & 0x80000000u) | ((e + 896u) << 20) | ((b & 0x7FFFFFu) >> 3);
  return e == 0u ? 0.0 : __hiloint2double((int)hi, (int)(b << 29));
}
__device__ __forceinline__ void seed_nb(float r2e, double &y0, double &t, bool &ok) {
  float y0f;
  seed_nb(r2e, y0, t, ok, y0f);
}
__device__ __forceinline__ bool seed_est(float r2e, double &y0, double &t) {
  bool ok;
  seed_nb(r2e, y0, t, ok);
  return ok;
}
// 1/sqrt(r2): y0 (1 + e/2 + 3e^2/8).  Every lane of the warp must call it.
__device__ __forceinline__ double rsq_est(double r2, float r2e) {
  double y0 = 0.0, t = 0.0;
  if (__all_sync(FULL, seed_est(r2e, y0, t))) {
    const double e = fma(-r2, t, 1.0);
    return fma(y0 * e, fma(e, 0.375, 0.5), y0);
  }
  return rsqrt(r2);
}
// Branch-free forms for the straight common sub-step (a branch would end the block the
// scheduler interleaves): ok reports whether the seed was in range; the caller votes on it and
// takes the forms above when any lane was not.
//
// The correction y0 + e (y0/2 + e 3y0/8) takes three FP64 instructions: y0/2 and 3y0/8 are exact
// (a 24-bit significand times 3 fits) and built from the seed's bits on the integer pipe, before
// r2 -- which the FP64 instructions wait for -- is ready.
__device__ __forceinline__ double rsq_nb(double r2, float r2e, bool &ok) {
  double y0, t;
  float y0f;
  seed_nb(r2e, y0, t, ok, y0f);
  const unsigned b = __float_as_uint(y0f);
  const double y0h = __longlong_as_double(__double_as_longlong(y0) - (1ll << 52));      // y0 / 2
  const double y038 = u64_scaled(3ull * ((b & 0x7FFFFFu) | 0x800000u),               // 3 y0 / 8
                                 (int)((b >> 23) & 0xFFu) - 153);
  const double e = fma(-r2, t, 1.0);
  return fma(e, fma(e, y038, y0h), y0);
}
// r2^(-3/2) = y0^3 (1 - e)^(-3/2) = y0^3 (1 + 3e/2 + 15e^2/8) to e^3 ~ 2^-62, with y0^3 = t y0;
// also t and e, from which 1/r2 = t (1 + e + e^2).  Every lane of the warp must call it.
__device__ __forceinline__ double rinv3_est(double r2, float r2e, double &t, double &e) {
  double y0 = 0.0;
  if (__all_sync(FULL, seed_est(r2e, y0, t))) {
    e = fma(-r2, t, 1.0);
    const double ty0 = t * y0;
    return fma(ty0, e * fma(e, 1.875, 1.5), ty0);
  }
  const double ri = rsqrt(r2);
  t = ri * ri;
  e = 0.0;
  return t * ri;
}


// per-level constants of the single-pair path, cached in shared memory
enum {
  LC_H, LC_HH, LC_T2, LC_R2, LC_A1, LC_B1, LC_A2, LC_B2, LC_GHA, LC_GHB, LC_T3, LC_MUNH, LC_H15,
  LC_R2N, LC_R2P, LC_N
};

// Runs the sub-steps of levels >= k with F_{k-1} = {q}, from the opening of a sub-step at level
// k.  X, V: this lane's component (packed layout).  Returns 0 when level k has finished (k is then
// k - 1), 1 when the pair may be in contact at the next check (k is that check's level; the
// general path takes the sub-step), 2 when the sub-step budget ran out.
__device__ __noinline__ int pair_run(const Dev &D, const GroupCtx &C, int lane, double *hs, int *cs,
                                     double *lc, double &Xio, double &Vio, double gA, double gB,
                                     double pR0sq, double piR0, double pRcut, int &kio, int &plev_io,
                                     long long &substeps_io, int &deepest_io) {
  const int pc = lane & 3, pb = (lane >> 2) & 1, cp = lane >> 3, base = lane & ~3;
  const unsigned m0 = (cp & 1) ? 0xffffffffu : 0u, m1 = (cp & 2) ? 0xffffffffu : 0u;
  // the two packed stages of the shell weight, with their copy-dependent constants set once:
  // stage1 = [x^2 | 70 - 20 x | 35 - 84 x | 1/r^2], stage2 = [+-x^4 | x^2 qa + qb | 1/r^3 | +-x^4]
  const unsigned mc0 = cp == 0 ? 0xffffffffu : 0u, mc1 = cp == 1 ? 0xffffffffu : 0u;
  const unsigned mc2 = cp == 2 ? 0xffffffffu : 0u, mc3 = cp == 3 ? 0xffffffffu : 0u;
  const double kb1 = cp == 1 ? -20.0 : -84.0, kc1 = cp == 1 ? 70.0 : (cp == 2 ? 35.0 : -0.0);
  const double kd3 = cp == 1 ? -0.5 : -1.0 / 6.0;
  auto stage1 = [&](double xw, double ri) {
    return fma_rn(bsel(ri, xw, mc3), bsel(xw, bsel(ri, kb1, mc3), mc0), kc1);
  };
  auto stage2 = [&](double x2s, double x2, double qa, double qb, double ri2, double ri) {
    return fma_rn(bsel(ri2, bsel(x2, x2s, mc1), mc2), bsel(ri, bsel(qa, x2, mc1), mc2),
                  bsel(qb, -0.0, mc1));
  };
  const unsigned mb = pb ? 0xffffffffu : 0u;
  const long long sgn_a = pb ? 0ll : (long long)0x8000000000000000ull;    // sign flip on body a
  const long long sgn_b = pb ? (long long)0x8000000000000000ull : 0ll;    // and on body b
  auto flip = [](double v, long long s) { return __longlong_as_double(__double_as_longlong(v) ^ s); };
  const DiskDesc *dp = C.dp;
  const double mu = C.mu;
  // group constants in registers (the loop stores through hs and cs, which could alias C)
  const int cM = C.M, cmax_sub = C.max_substeps, cmax_depth = C.max_depth, cd = C.d;
  const double c_invM = C.invM;
  const bool c_pow2 = (cM & (cM - 1)) == 0;
  const float muf = f32_trunc(mu);
  double X = Xio, V = Vio;
  long long substeps = substeps_io;
  int deepest = deepest_io, plev = plev_io;
  const int k0 = kio;
  int j = k0, cj = cs[j];
  unsigned long long have = 0ull;

  // current level's constants
  // (h^2, h^3 and 1.5 h serve only the order-3 drift, which reads them from the cache)
  double h, hh, R2, A1, B1, A2, B2, ghs, munh, R2n, R2p;
  float hf, R2f;
  auto set_level = [&](int jj) {
    double *Lc = lc + LC_N * jj;
    if (!((have >> jj) & 1ull)) {
      const double hj = hs[jj];
      // [h/2 | h^2 | R_j^2 | R_{j+1}^2]
      const double s1 = fma4(m0, m1, hj, 0.5, -0.0, hj, hj, -0.0, pR0sq, dp->ck2[jj], -0.0,
                             pR0sq, dp->ck2[jj + 1], -0.0);
      const double hh_ = cpy(s1, lane, 0), t2_ = cpy(s1, lane, 1);
      // weight argument (r - R_{j+1}) / (R_j - R_{j+1}) = r A1 + B1, and the same one level up
      const double s2 = fma4(m0, m1, piR0, dp->invdc[jj], -0.0, dp->ck[jj + 1], dp->invdc[jj], -0.0,
                             piR0, dp->invdc[jj - 1], -0.0, dp->ck[jj], dp->invdc[jj - 1], -0.0);
      // [G m_a h/2 | G m_b h/2 | h^3 | -mu h]
      const double s3 = fma4(m0, m1, gA, hh_, -0.0, gB, hh_, -0.0, t2_, hj, -0.0, mu, -hj, -0.0);
      // [mu h/2 | 1.5 h | R_{j-1}^2]; -mu h times the series coefficients of r^-3 below
      const double s4 = fma4(m0, m1, mu, hh_, -0.0, hh_, 1.0, hj, pR0sq, dp->ck2[jj - 1], -0.0,
                             mu, hh_, -0.0);
      const double v[LC_N] = {hj, hh_, t2_, cpy(s1, lane, 2), cpy(s2, lane, 0), -cpy(s2, lane, 1),
                              cpy(s2, lane, 2), -cpy(s2, lane, 3), cpy(s3, lane, 0),
                              cpy(s3, lane, 1), cpy(s3, lane, 2), cpy(s3, lane, 3), cpy(s4, lane, 1),
                              cpy(s1, lane, 3), cpy(s4, lane, 2)};
#pragma unroll
      for (int i = 0; i < LC_N; ++i) Lc[i] = v[i];
      have |= 1ull << jj;
    }
    h = Lc[LC_H]; hh = Lc[LC_HH]; R2 = Lc[LC_R2];
    A1 = Lc[LC_A1]; B1 = Lc[LC_B1]; A2 = Lc[LC_A2]; B2 = Lc[LC_B2];
    ghs = flip(Lc[pb ? LC_GHA : LC_GHB], sgn_b);       // -G m_a h/2 on body b, G m_b h/2 on a
    munh = Lc[LC_MUNH];
    R2n = Lc[LC_R2N]; R2p = Lc[LC_R2P];
    hf = f32_trunc(h);
    R2f = f32_trunc(R2) * (1.0f + 3.0517578e-5f);     // not below R2
  };

  // separation x_b - x_a (this lane's component), its square norm, and that in FP32 (not above)
  double d = 0.0, r2 = 0.0;
  float r2f = 0.0f, r2e = 0.0f;
  double c_ri = 0.0, c_ri3 = 0.0, c_f = 0.0;
  bool rcache = false;          // c_ri, c_ri3 hold 1/r and 1/r^3 of the current positions
  int c_lvl = -1;               // level of the last force at these positions, its weight c_f,
  bool c_inner = false;         // and whether that weight was g (inside R_level, non-zero)
  bool c_outer = false;         // or 1 - g of the level above (outside R_level, non-zero)
  // (Xo: the other body's x in this lane's copy and component)
  auto sep2 = [&](double Xo) {
    // x_b - x_a on both bodies' lanes as a sum of sign-flipped operands (exactly X - Xo, Xo - X)
    d = flip(X, sgn_a) + flip(Xo, sgn_b);
    const float df = f32_trunc(d);
    const float a = __shfl_sync(FULL, df, base), b = __shfl_sync(FULL, df, base + 1);
    const float c = __shfl_sync(FULL, df, base + 2);
    r2e = fmaf(c, c, fmaf(b, b, a * a));        // FP32 estimate: seeds 1/r before r2 is formed
    r2 = csum3(d * d, base);
    r2f = f32_trunc(r2);
    rcache = false;
  };
  auto sep = [&]() { sep2(__shfl_xor_sync(FULL, X, 4)); };

  // level-j force: hc = (h/2) w_j(r) G m_other / r^3 with this body's sign, zero when w_j
  // vanishes (fz: outside [R_{j+1}, R_{j-1})).  Branch-free, so that it schedules together with
  // the work around it; forces_skip() leaves it out when the weight vanishes.
  double hc = 0.0;
  bool fz = true;
  auto forces = [&]() {
    fz = lt_nn(r2, R2n) || !lt_nn(r2, R2p);
    const bool inner = lt_nn(r2, R2);        // w_j = g_j inside R_j, 1 - g_{j-1} outside
    // the weight's level constants, chosen by bit selects (no branch): A, B from shell j
    // (inside R_j) or j - 1, zero with g when the weight vanishes
    const unsigned m_in = inner ? 0xffffffffu : 0u, m_fz = fz ? 0xffffffffu : 0u;
    const double A = bsel(0.0, bsel(A1, A2, m_in), m_fz), B = bsel(0.0, bsel(B1, B2, m_in), m_fz);
    const double g = bsel(0.0, ghs, m_fz);
    const long long s_out = inner ? 0ll : (long long)0x8000000000000000ull;   // sign of x^4
    if (rcache && c_lvl == j - 1 && c_inner && !inner && !fz) {
      // entering level j at the positions of the last level-(j-1) force, with the pair between
      // R_j and R_{j-1}: the weights telescope, w_j = 1 - g_{j-1}(r) = 1 - w_{j-1} (the same
      // argument (r - R_j) / (R_{j-1} - R_j) in both), so only the products remain
      const double wt = 1.0 - c_f;
      hc = wt * (c_ri3 * g);
      c_f = wt;
      c_lvl = j;
      c_inner = false;
      c_outer = true;
      return;
    }
    if (rcache && c_lvl == j + 1 && c_outer && inner && !fz) {
      // back at level j at the positions of the last level-(j+1) force, with the pair between
      // R_{j+1} and R_j: w_j = g_j(r) = 1 - w_{j+1} (the same argument (r - R_{j+1}) /
      // (R_j - R_{j+1}) in both)
      const double wt = 1.0 - c_f;
      hc = wt * (c_ri3 * g);
      c_f = wt;
      c_lvl = j;
      c_inner = true;
      c_outer = false;
      return;
    }
    // 1/r and 1/r^3 are level-independent: on entering a deeper level at unchanged positions
    // the last ones are reused and only the weight is new.  The weight argument r A + B is
    // formed as (1/r)(r^2 A) + B, so that r^2 A is ready before the reciprocal square root.
    const double ri = rcache ? c_ri : rsq_est(r2, r2e);
    const double xw = fma(ri, r2 * A, B);
    // f_3(x) = x^4 ((35 - 84 x) + x^2 (70 - 20 x)):  [x^2 | 70 - 20 x | 35 - 84 x | 1/r^2]
    const double s1 = stage1(xw, ri);
    const double x2 = cpy(s1, lane, 0), qa = cpy(s1, lane, 1), qb = cpy(s1, lane, 2);
    const double ri2 = cpy(s1, lane, 3);
    // [+-x^4 | x^2 qa + qb | 1/r^3]  (the sign of x^4 picks f or 1 - f)
    const double x2s = flip(x2, s_out);
    const double s2 = stage2(x2s, x2, qa, qb, ri2, ri);
    const double x4s = cpy(s2, lane, 0), q = cpy(s2, lane, 1);
    const double ri3 = bsel(c_ri3, cpy(s2, lane, 2), rcache ? 0xffffffffu : 0u);
    c_ri = ri;
    c_ri3 = ri3;
    rcache = true;
    // no clamp of x to [0, 1]: outside [R_{j+1}, R_{j-1}) the weight is zero (fz, x = 0 above),
    // inside x leaves [0, 1] only by rounding, where f_3 (flat at both ends) differs from 0 or
    // 1 by O(x^4) or O((x - 1)^2)
    const double w = fma(x4s, q, bsel(-0.0, 1.0, m_in));
    hc = w * (ri3 * g);
    c_f = w;
    c_lvl = j;
    c_inner = inner && !fz;
    c_outer = !inner && !fz;
  };
  // the same for the straight block: no branch; f_ok = false when the seed was out of range
  bool f_ok = true;
  auto forces_nb = [&]() {
    fz = lt_nn(r2, R2n) || !lt_nn(r2, R2p);
    const bool inner = lt_nn(r2, R2);
    // the weight's level constants, chosen by bit selects (no branch): A, B from shell j
    // (inside R_j) or j - 1, zero with g when the weight vanishes
    const unsigned m_in = inner ? 0xffffffffu : 0u, m_fz = fz ? 0xffffffffu : 0u;
    const double A = bsel(0.0, bsel(A1, A2, m_in), m_fz), B = bsel(0.0, bsel(B1, B2, m_in), m_fz);
    const double g = bsel(0.0, ghs, m_fz);
    const long long s_out = inner ? 0ll : (long long)0x8000000000000000ull;   // sign of x^4
    bool ok;
    const double ri = rsq_nb(r2, r2e, ok);
    f_ok = __all_sync(FULL, ok);
    const double xw = fma(ri, r2 * A, B);
    const double s1 = stage1(xw, ri);
    const double x2 = cpy(s1, lane, 0), qa = cpy(s1, lane, 1), qb = cpy(s1, lane, 2);
    const double ri2 = cpy(s1, lane, 3);
    const double x2s = flip(x2, s_out);
    const double s2 = stage2(x2s, x2, qa, qb, ri2, ri);
    const double x4s = cpy(s2, lane, 0), q = cpy(s2, lane, 1), ri3 = cpy(s2, lane, 2);
    const double w = fma(x4s, q, bsel(-0.0, 1.0, m_in));
    hc = w * (ri3 * g);
    c_ri = ri;
    c_ri3 = ri3;
    c_f = w;
    c_lvl = j;
    c_inner = inner && !fz;
    c_outer = !inner && !fz;
    rcache = f_ok;
  };
  auto forces_skip = [&]() {
    fz = lt_nn(r2, R2n) || !lt_nn(r2, R2p);
    if (fz) { hc = 0.0; return; }
    forces();
  };

  // (i): minimum distance of the straight-line relative motion over [0, h] below R_j, for the
  // velocities U (before this sub-step's opening kick).  far_apart() is a conservative FP32 test
  // of the common case, |d| - |dv| h > R_j, with relative margins of 2^-15, far above the
  // rounding of its FP32 copies (truncation 2^-23 per operand), so it never clears a pair the
  // FP64 predicate would flag; check_exact() is the FP64 predicate.
  auto far_apart = [&](double U) -> bool {
    const float uf = f32_trunc(U), uo = __shfl_xor_sync(FULL, uf, 4);
    // u_b - u_a on both bodies' lanes (only its square is used)
    const float dvf = __uint_as_float(__float_as_uint(uf - uo) ^ (pb ? 0u : 0x80000000u));
    const float av = fabsf(uf) + fabsf(uo);
    const float p0 = dvf * dvf;
    const float s2 = (__shfl_sync(FULL, p0, base) + __shfl_sync(FULL, p0, base + 1)) +
                     __shfl_sync(FULL, p0, base + 2);
    const float sa = (__shfl_sync(FULL, av, base) + __shfl_sync(FULL, av, base + 1)) +
                     __shfl_sync(FULL, av, base + 2);
    const float m = 1.0f + 3.0517578e-5f;                       // 1 + 2^-15
    // square roots as x rsqrt(x) (relative error below 2^-21, inside the margins; x = 0 gives
    // NaN, which fails the test)
    const float dvmag = s2 * rsqrtf(s2) * m + sa * 2.3841858e-7f;   // |dv| + truncation error (2^-22)
    const float dlo = r2f * rsqrtf(r2f) * (1.0f - 3.0517578e-5f);
    const float rhs = (R2f * rsqrtf(R2f) + dvmag * hf * m) * m;
    return R2f > 0.0f && dlo > rhs;                             // NaN and underflow: false
  };
  auto check_exact = [&](double U) -> bool {
    if (lt_nn(r2, R2)) return true;
    const double Uo = __shfl_xor_sync(FULL, U, 4);
    const double dv = bsel(U, Uo, mb) - bsel(Uo, U, mb);
    const double vr = csum3(d * dv, base), v2 = csum3(dv * dv, base);
    if (!is_neg(vr)) return false;
    // [h v2 | vr^2 | R2 v2 | 2 vr]
    const double s = fma4(m0, m1, h, v2, -0.0, vr, vr, -0.0, R2, v2, -0.0, vr, 2.0, -0.0);
    const double hv2 = cpy(s, lane, 0);
    if (lt_nn(neg(vr), hv2)) return lt_nn(fma(r2, v2, -cpy(s, lane, 1)), cpy(s, lane, 2));
    const double e = fma(h, fma(h, v2, cpy(s, lane, 3)), r2);
    return is_neg(e) || lt_nn(e, R2);
  };

  // distance of this lane's body from the sun at the current positions (1/r^3, and the pieces
  // of 1/r^2), computed at the opening of a sub-step, where it overlaps the FP32 decisions
  // 1/r^3; 1/r^2 = rbt (1 + rbe + rbe^2); body_r_nb() leaves rb3 to rb3_nb() and keeps rbty =
  // y0^3 = rbt y0, so that 1/r^3 = rbty (1 + 3e/2 + 15e^2/8) with e = rbe
  double rb3 = 0.0, rbt = 0.0, rbe = 0.0, rbty = 0.0;
  bool rb_ok = true;
  auto body_r = [&]() {
    const float xf = f32_trunc(X);
    const float a = __shfl_sync(FULL, xf, base), b = __shfl_sync(FULL, xf, base + 1);
    const float c = __shfl_sync(FULL, xf, base + 2);
    const float rbf2 = fmaf(c, c, fmaf(b, b, a * a));
    rb3 = rinv3_est(csum3(X * X, base), rbf2, rbt, rbe);
    rb_ok = true;
  };
  float bx0 = 0.0f, bx1 = 0.0f, bx2 = 0.0f, brif = 0.0f;   // FP32 copies of x and 1/|x| (seed)
  auto body_r_nb = [&]() {                  // branch-free; rb_ok = false: take body_r()
    const float xf = f32_trunc(X);
    bx0 = __shfl_sync(FULL, xf, base);
    bx1 = __shfl_sync(FULL, xf, base + 1);
    bx2 = __shfl_sync(FULL, xf, base + 2);
    const float rbf2 = fmaf(bx2, bx2, fmaf(bx1, bx1, bx0 * bx0));
    const double rs2 = csum3(X * X, base);
    double y0;
    bool ok;
    seed_nb(rbf2, y0, rbt, ok, brif);
    rbe = fma(-rs2, rbt, 1.0);
    rbty = rbt * y0;
    rb_ok = __all_sync(FULL, ok);
  };
  auto rb3_nb = [&]() { rb3 = fma(rbty, rbe * fma(rbe, 1.875, 1.5), rbty); };
  // the FP64 part of body_r_nb() from the seed body_f32() took (valid when rb_ok)
  auto body_r64 = [&]() {
    const double rs2 = csum3(X * X, base);
    double y0;
    seed_expand(brif, y0, rbt);
    rbe = fma(-rs2, rbt, 1.0);
    rbty = rbt * y0;
  };
  // the FP32 part of body_r_nb() alone: the copies of x and the seed 1/|x| the FP32 decisions use
  auto body_f32 = [&]() {
    const float xf = f32_trunc(X);
    bx0 = __shfl_sync(FULL, xf, base);
    bx1 = __shfl_sync(FULL, xf, base + 1);
    bx2 = __shfl_sync(FULL, xf, base + 2);
    bool ok;
    seed_f32(fmaf(bx2, bx2, fmaf(bx1, bx1, bx0 * bx0)), ok, brif);
    rb_ok = __all_sync(FULL, ok);
  };
  // 1/r^3 of this lane's body, carried along the common sub-steps: a common sub-step drifts by
  // the order-2 series, which moves r^2 by the factor 1 + u with
  //   u = 2 h (x.v)/r^2 + h^2 (v^2/r^2 - mu/r^3)  (+ h^3 mu (x.v)/r^5 and smaller),
  // so 1/r^3 moves by (1 + u)^(-3/2) = 1 - 3u/2 + 15u^2/8 (+ O(u^3)).  The order-2 regime bounds
  // h^2 max(mu/r^3, ((x.v)/r^2)^2, |v^2/r^2 - mu/r^3|) by 5e-13, so |u| < 2e-6, the dropped
  // terms are below 1e-18, and the FP32 evaluation of u from the decisions' truncated copies
  // errs by at most ~1e-12 (2^-39.7) relative per sub-step.  After GC_MAX carried sub-steps
  // (2^-34.7 at most) 1/r^3 is formed again in full.  f' = -mu h/r^3 enters v' as f' x, which
  // in the order-2 regime is below 7e-7 of v on a bound orbit, so the carried factor moves v
  // by less than 2^-55 of v.
  constexpr int GC_MAX = 32;
  double rb3c = 0.0;
  int gc_n = GC_MAX;            // carried sub-steps since 1/r^3 was formed; GC_MAX: not valid

  // u = mu/r^3, p = (x.v)/r^2 and q = v^2/r^2 - u of this lane's body in FP32, from the last
  // order decision: the drift series take from them the terms whose size bounds their needed
  // precision far below FP32's (f' (3/2) p h for order 2, the t^3 term of f' for order 3)
  float ds_u = 0.0f, ds_p = 0.0f, ds_q = 0.0f;
  // order of the drift series for both bodies over h, from FP32 copies (the thresholds of
  // drift_series): 2, 3, 6, or 9 for the Kepler solver
  auto drift_order = [&]() -> unsigned {
    const float xf = f32_trunc(X), vf = f32_trunc(V);
    const float x0 = __shfl_sync(FULL, xf, base), x1 = __shfl_sync(FULL, xf, base + 1);
    const float x2f = __shfl_sync(FULL, xf, base + 2);
    const float v0 = __shfl_sync(FULL, vf, base), v1 = __shfl_sync(FULL, vf, base + 1);
    const float v2f = __shfl_sync(FULL, vf, base + 2);
    const float rrf = fmaf(x2f, x2f, fmaf(x1, x1, x0 * x0));
    const float rvf = fmaf(x2f, v2f, fmaf(x1, v1, x0 * v0));
    const float vvf = fmaf(v2f, v2f, fmaf(v1, v1, v0 * v0));
    const float rif = rsqrtf(rrf), ri2f = rif * rif;
    const float uf = muf * ri2f * rif, pf = rvf * ri2f, qf = fmaf(vvf, ri2f, -uf);
    const float so = fmaxf(fmaxf(uf, pf * pf), fabsf(qf)) * hf * hf;
    ds_u = uf;
    ds_p = pf;
    ds_q = qf;
    return __reduce_max_sync(FULL, !(so <= 2.0e-6f) ? 9u : (so < 5e-13f ? 2u : (so < 5e-10f ? 3u : 6u)));
  };
  // the same decision from the FP32 copies and the seed body_r_nb() took (valid when rb_ok)
  auto drift_order_nb = [&](float &pfo, float &qfo) -> unsigned {
    const float vf = f32_trunc(V);
    const float v0 = __shfl_sync(FULL, vf, base), v1 = __shfl_sync(FULL, vf, base + 1);
    const float v2f = __shfl_sync(FULL, vf, base + 2);
    const float rvf = fmaf(bx2, v2f, fmaf(bx1, v1, bx0 * v0));
    const float vvf = fmaf(v2f, v2f, fmaf(v1, v1, v0 * v0));
    const float ri2f = brif * brif;
    const float uf = muf * ri2f * brif, pf = rvf * ri2f, qf = fmaf(vvf, ri2f, -uf);
    const float so = fmaxf(fmaxf(uf, pf * pf), fabsf(qf)) * hf * hf;
    pfo = pf;
    qfo = qf;
    ds_u = uf;
    ds_p = pf;
    ds_q = qf;
    return __reduce_max_sync(FULL, !(so <= 2.0e-6f) ? 9u : (so < 5e-13f ? 2u : (so < 5e-10f ? 3u : 6u)));
  };

  // Kepler drift of both bodies over h: Lagrange series of order 2 or 3, else the scalar path
  auto drift = [&](unsigned ord) {
    if (ord == 2u) {
      // f - 1 = f' h/2 with f' = -mu h/r^3: x' = (x + h/2 v) + h/2 (v + f' x), v' = v + f'' Y with
      // f'' = f' (1 - 3/2 p h), the series' f' to second order (a term of up to 1e-6 of f', which
      // moves v by up to 7e-13 of v; its FP32 evaluation errs by < 1e-18 of v)
      const double fd = munh * rb3;
      const double W = fma(fd, X, V), Y = fma(hh, V, X);
      X = fma(hh, W, Y);
      V = fma(fma(fd, f32_to_f64(-1.5f * hf * ds_p), fd), Y, V);
    } else if (ord == 3u) {
      const double X1 = fma(h, V, X);
      const double rv = csum3(X * V, base);
      const double rb2 = fma(rbt, fma(rbe, rbe, rbe), rbt);
      const double u = mu * rb3, p = rv * rb2;
      // [u p | -u/2 | -u/6 | u p]
      const double s3 = u * bsel(kd3, p, mc1 | mc2);
      const double up = cpy(s3, lane, 0), nhu = cpy(s3, lane, 1), nu6 = cpy(s3, lane, 2);
      // [h/2 up - u/2 | 1.5 h up - u | h up - u/2 | -u h^3/6]
      // h^2, h^3 and 1.5 h from the level cache (needed only here)
      const double *Lc = lc + LC_N * j;
      const double t2 = Lc[LC_T2], t3 = Lc[LC_T3], h15 = Lc[LC_H15];
      const double s4 = fma4(m0, m1, hh, up, nhu, h15, up, -u, h, up, nhu, t3, nu6, -0.0);
      // [f - 1 | f' | g' - 1 | x + h v + (g - h) v]
      // f' to third order: + (3uq - 15up^2 + u^2) h^3/6, below 3.3e-14 of v in the order-3 regime,
      // so its FP32 evaluation suffices
      const float hk3 = (3.0f * ds_u * ds_q - 15.0f * ds_u * ds_p * ds_p + ds_u * ds_u) *
                        (1.0f / 6.0f) * hf * hf * hf;
      const double s5 = fma4(m0, m1, t2, cpy(s4, lane, 0), -0.0, h, cpy(s4, lane, 1),
                             f32_to_f64(hk3), t2, cpy(s4, lane, 2), -0.0, cpy(s4, lane, 3), V, X1);
      const double fm1 = cpy(s5, lane, 0), fd = cpy(s5, lane, 1), gdm1 = cpy(s5, lane, 2);
      const double Xn = fma(fm1, X, cpy(s5, lane, 3));
      V = fma(fd, X, fma(gdm1, V, V));
      X = Xn;
    } else {
      // longer intervals: the scalar series of order 6 or the Kepler solver, per body, in every
      // lane of the body
      double bx = SH(X, base), by = SH(X, base + 1), bz = SH(X, base + 2);
      double bvx = SH(V, base), bvy = SH(V, base + 1), bvz = SH(V, base + 2);
      if (!drift_series(mu, h, bx, by, bz, bvx, bvy, bvz)) {
        const int st = kepler_drift(mu, h, bx, by, bz, bvx, bvy, bvz);
        if (st != SYMBA_OK && pc == 0 && cp == 0) set_status(&D.stat[cd], st);
      }
      __syncwarp();
      X = pc == 0 ? bx : (pc == 1 ? by : (pc == 2 ? bz : 0.0));
      V = pc == 0 ? bvx : (pc == 1 ? bvy : (pc == 2 ? bvz : 0.0));
    }
  };

  int rc = 0;
  int fat = -1;                 // level of the forces held in hc
  bool start = true;
  set_level(j);
  sep();
  deepest = max(deepest, j);
  for (;;) {
    bool level_done = false;
    if (start) {
      {
        // the rare cases of a sub-step's opening under one branch: contact possible, budget
        // spent, or the forces held are another level's
        const bool touch = lt_nn(r2, pRcut), over = substeps >= cmax_sub;
        if (touch || over || fat != j) {
          if (touch || over) {
            if (touch) {
              rc = 1;
            } else {
              ++substeps;
              rc = 2;
            }
            break;
          }
          forces_skip();
          fat = j;
        }
      }
      ++substeps;
      const double U = V;                  // velocities the check sees
      V = fma(hc, d, V);                   // opening kick (hc = 0 when the weight vanishes)
      bool fl = lt_nn(r2, R2);             // inside R_j: the pair is in F_j
      if (!fl) {
        // one straight block: the FP32 decisions and the order-2 drift they usually select, with
        // 1/r^3 carried (rb3c); when it is not valid, the sub-step takes the forms below
        body_f32();
        const bool far = far_apart(U);
        float pf, qf;
        unsigned ord = drift_order_nb(pf, qf);
        // the order-2 drift as in drift(2): copies 0-1 form W = f' x + v and then x' = h/2 W + Y,
        // copies 2-3 Y = h/2 v + x and then v' = f'' Y + v, with f' = -mu h/r^3 and
        // f'' = f' (1 - 3/2 p h), the series' f' to second order
        const double fd = munh * rb3c;
        const double fdv = fma(fd, f32_to_f64(-1.5f * hf * pf), fd);
        const double s_wy = fma_rn(bsel(hh, fd, m1), bsel(V, X, m1), bsel(X, V, m1));
        const double W = cpy(s_wy, lane, 0), Y = cpy(s_wy, lane, 2);
        const double s_xv = fma_rn(bsel(fdv, hh, m1), bsel(Y, W, m1), bsel(V, Y, m1));
        const double Xn = cpy(s_xv, lane, 0), Vn = cpy(s_xv, lane, 2);
        const double Xno = __shfl_sync(FULL, s_xv, (lane & 7) ^ 4);     // the other body's x'
        // (1 + u)^(-3/2) - 1 for this drift (valid with the order-2 series and rb_ok)
        const float u = fmaf(2.0f * hf, pf, hf * hf * qf);
        const double dr3 = f32_to_f64(u * fmaf(1.875f, u, -1.5f));
        if (far && ord == 2u && rb_ok && gc_n < GC_MAX) {
          // the common sub-step: F_j stays empty, series of order 2, closing force and kick
          plev = j - 1;
          X = Xn;
          V = Vn;
          rb3c = fma(rb3c, dr3, rb3c);
          ++gc_n;
          sep2(Xno);
          const double Vk = V;
          forces_nb();
          V = fma(hc, d, Vk);
          if (!f_ok) {                      // a seed out of range: the general form
            forces();
            V = fma(hc, d, Vk);
          }
          fat = j;
          if (++cj < cM) continue;
          level_done = true;
        } else {
          // 1/r^3 in full; an order-2 drift from here starts a new carried run
          const bool fresh = far && ord == 2u && rb_ok;
          if (rb_ok) {
            body_r64();
            rb3_nb();
          } else {
            body_r();
            ord = drift_order();
          }
          gc_n = GC_MAX;
          if (fresh) {
            rb3c = fma(rb3, dr3, rb3);
            gc_n = 0;
          }
          if (far && ord <= 3u) {
            plev = j - 1;
            drift(ord);
            sep();
            forces_nb();
            if (!f_ok) forces();
            V = fma(hc, d, V);
            fat = j;
            if (++cj < cM) continue;
            level_done = true;
          } else {
            fl = !far && check_exact(U);
            if (!fl) {
              plev = j - 1;
              drift(ord);
              sep();
              start = false;
            }
          }
        }
      }
      if (fl) {
        plev = j;
        if (j + 1 <= cmax_depth) {
          cs[j] = cj;
          ++j;
          deepest = max(deepest, j);          // a level is entered only here (and at the start)
          hs[j] = c_pow2 ? hs[j - 1] * c_invM : hs[j - 1] / (double)cM;
          cj = 0;
          set_level(j);
          continue;
        }
        if (lane == 0) set_status(&D.stat[cd], SYMBA_E_DEPTH);
        body_r();
        drift(drift_order());
        gc_n = GC_MAX;
        sep();
        start = false;
      }
    }
    if (!level_done) {
      forces_skip();
      fat = j;
      if (!fz) V = fma(hc, d, V);
      if (++cj < cM) { start = true; continue; }
    }
    --j;
    fat = -1;
    start = false;
    if (j < k0) break;
    cj = cs[j];
    set_level(j);
  }
  if (j >= k0) cs[j] = cj;
  kio = j;
  Xio = X;
  Vio = V;
  substeps_io = substeps;
  deepest_io = deepest;
  plev_io = plev;
  return rc;
}

__device__ void run_group_regs(const Dev &D, const GroupCtx &C, int lane, double *hs, int *cs, double *lc) {
  const int nm = C.mcnt, np = C.pcnt;
  const bool ism = lane < nm, isp = lane < np;
  // bodies
  int pglob = -1;
  double x = 0.0, y = 0.0, z = 0.0, vx = 0.0, vy = 0.0, vz = 0.0, m = 0.0, gm = 0.0, rad = 0.0, rh = 0.0;
  int alive = 0;
  if (ism) {
    pglob = D.gmem[C.moff + lane];
    x = D.x[pglob]; y = D.y[pglob]; z = D.z[pglob];
    vx = D.vx[pglob]; vy = D.vy[pglob]; vz = D.vz[pglob];
    m = D.m[pglob]; gm = D.gm[pglob]; rad = D.rad[pglob]; rh = D.rh[pglob];
    alive = D.alive[pglob];
    D.mslot[pglob] = lane;
  }
  __syncwarp();
  // pairs
  int ia = 0, ib = 0, lev = -1;
  if (isp) {
    ia = D.mslot[D.gpi[C.poff + lane]];
    ib = D.mslot[D.gpj[C.poff + lane]];
    lev = 0;
  }
  // per-pair constants: critical radius R_0, 1/R_0, R_0^2 and the contact prefilter threshold
  double R0, iR0, R0sq, Rcut;
  auto pair_consts = [&]() {
    const double ra = SH(rh, ia), rb = SH(rh, ib);
    const double sa = SH(rad, ia), sb = SH(rad, ib);
    R0 = __dmul_rn(C.lam, __dadd_rn(ra, rb));
    iR0 = R0 > 0.0 ? 1.0 / R0 : 0.0;
    R0sq = R0 * R0;
    const double Rc = sa + sb;
    Rcut = 1.0000001 * (Rc * Rc);
  };
  pair_consts();
  unsigned im = 0u, jm = 0u;
  for (int q = 0; q < np; ++q) {
    const int a_ = SH(ia, q), b_ = SH(ib, q);
    if (a_ == lane) im |= 1u << q;
    if (b_ == lane) jm |= 1u << q;
  }
  const unsigned adjm = ism ? (im | jm) : 0u;
  double fdx = 0.0, fdy = 0.0, fdz = 0.0, ffi = 0.0, ffj = 0.0;   // forces of pair `lane`

  auto forces = [&](int k) {
    const unsigned Lm = __ballot_sync(FULL, isp && lev >= k - 1);
    const double xa = SH(x, ia), ya = SH(y, ia), za = SH(z, ia);
    const double xb = SH(x, ib), yb = SH(y, ib), zb = SH(z, ib);
    const double ga = SH(gm, ia), gb = SH(gm, ib);
    const int aa = SH(alive, ia), ab = SH(alive, ib);
    fdx = fdy = fdz = ffi = ffj = 0.0;
    if (((Lm >> lane) & 1u) && aa && ab) {
      fdx = xb - xa; fdy = yb - ya; fdz = zb - za;
      const double r2 = fma(fdz, fdz, fma(fdy, fdy, fdx * fdx));
      const double ri = rsqrt_fp64(r2);
      const double rho = r2 * ri * iR0;
      const double ck = C.dp->ck[k], ck1 = C.dp->ck[k + 1];
      double w;
      if (k == 0 || lt_nn(rho, ck)) w = partition_fn((rho - ck1) * C.dp->invdc[k], C.l);
      else w = 1.0 - partition_fn((rho - ck) * C.dp->invdc[k - 1], C.l);
      const double s = w * (ri * ri * ri);
      ffi = gb * s;
      ffj = ga * s;
    }
  };

  auto kick = [&](int k, double hh) {
    const unsigned Lm = __ballot_sync(FULL, isp && lev >= k - 1);
    unsigned mine = adjm & Lm;
    const bool inS = mine != 0u;
    const int iters = __reduce_max_sync(FULL, (unsigned)__popc(mine));
    double ax = 0.0, ay = 0.0, az = 0.0;
    for (int it = 0; it < iters; ++it) {
      const int q = mine ? (__ffs(mine) - 1) : lane;
      const double qx = SH(fdx, q), qy = SH(fdy, q), qz = SH(fdz, q), qi = SH(ffi, q), qj = SH(ffj, q);
      if (mine) {
        const double f = ((im >> q) & 1u) ? qi : -qj;
        ax = fma(f, qx, ax); ay = fma(f, qy, ay); az = fma(f, qz, az);
        mine &= mine - 1u;
      }
    }
    if (inS && alive) {
      vx = fma(hh, ax, vx); vy = fma(hh, ay, vy); vz = fma(hh, az, vz);
    }
  };

  auto drift = [&](int k, double h, bool all) {
    const unsigned Lm = __ballot_sync(FULL, isp && lev >= k - 1);
    const unsigned Fm = __ballot_sync(FULL, isp && lev >= k);
    const bool inS = (adjm & Lm) != 0u, inF = (adjm & Fm) != 0u;
    if (alive && inS && (all || !inF)) {
      if (!drift_series(C.mu, h, x, y, z, vx, vy, vz)) {
        const int st = kepler_drift(C.mu, h, x, y, z, vx, vy, vz);
        if (st != SYMBA_OK) set_status(&D.stat[C.d], st);
      }
    }
  };

  // (i): returns whether F_k is non-empty; *merged when bodies merged
  auto check = [&](int k, double h, bool *merged) -> bool {
    const bool inL = isp && lev >= k - 1;
    const double xa = SH(x, ia), ya = SH(y, ia), za = SH(z, ia);
    const double xb = SH(x, ib), yb = SH(y, ib), zb = SH(z, ib);
    const int aa = SH(alive, ia), ab = SH(alive, ib);
    const double dx = xb - xa, dy = yb - ya, dz = zb - za;
    const double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
    const bool both = inL && aa && ab;
    const double rda = SH(rad, ia), rdb = SH(rad, ib);
    const bool ct = both && lt_nn(r2, Rcut) && contact_regs(xa, ya, za, xb, yb, zb, rda, rdb);
    if (!__any_sync(FULL, ct)) {
      const double vxa = SH(vx, ia), vya = SH(vy, ia), vza = SH(vz, ia);
      const double vxb = SH(vx, ib), vyb = SH(vy, ib), vzb = SH(vz, ib);
      bool fl = false;
      if (both) fl = predicate_regs(dx, dy, dz, r2, vxb - vxa, vyb - vya, vzb - vza, R0sq * C.dp->ck2[k], h);
      if (inL) lev = fl ? k : k - 1;
      *merged = false;
      return __any_sync(FULL, fl) != 0;
    }
    // mergers: the pairs one by one in list order, every lane following the same sequence
    bool nonempty = false;
    for (int q = 0; q < np; ++q) {
      if (SH(lev, q) < k - 1) continue;
      const int a_ = SH(ia, q), b_ = SH(ib, q);
      bool fl = false;
      if (SH(alive, a_) && SH(alive, b_)) {
        const double xa_ = SH(x, a_), ya_ = SH(y, a_), za_ = SH(z, a_);
        const double xb_ = SH(x, b_), yb_ = SH(y, b_), zb_ = SH(z, b_);
        const double ra_ = SH(rad, a_), rb_ = SH(rad, b_);
        const double vxa_ = SH(vx, a_), vya_ = SH(vy, a_), vza_ = SH(vz, a_);
        const double vxb_ = SH(vx, b_), vyb_ = SH(vy, b_), vzb_ = SH(vz, b_);
        const double ma = SH(m, a_), mb = SH(m, b_), rha = SH(rh, a_);
        if (contact_regs(xa_, ya_, za_, xb_, yb_, zb_, ra_, rb_)) {
          const double Mt = __dadd_rn(ma, mb);
          if (lane == a_) {
            if (Mt > 0.0) {
              x = __ddiv_rn(__dadd_rn(__dmul_rn(ma, xa_), __dmul_rn(mb, xb_)), Mt);
              y = __ddiv_rn(__dadd_rn(__dmul_rn(ma, ya_), __dmul_rn(mb, yb_)), Mt);
              z = __ddiv_rn(__dadd_rn(__dmul_rn(ma, za_), __dmul_rn(mb, zb_)), Mt);
              vx = __ddiv_rn(__dadd_rn(__dmul_rn(ma, vxa_), __dmul_rn(mb, vxb_)), Mt);
              vy = __ddiv_rn(__dadd_rn(__dmul_rn(ma, vya_), __dmul_rn(mb, vyb_)), Mt);
              vz = __ddiv_rn(__dadd_rn(__dmul_rn(ma, vza_), __dmul_rn(mb, vzb_)), Mt);
            }
            rad = cbrt_rn(__dadd_rn(__dmul_rn(__dmul_rn(ra_, ra_), ra_), __dmul_rn(__dmul_rn(rb_, rb_), rb_)));
            if (ma > 0.0) rh = __dmul_rn(rha, cbrt_rn(__ddiv_rn(Mt, ma)));
            m = Mt;
            gm = __dmul_rn(C.G, Mt);
          }
          if (lane == b_) { m = 0.0; gm = 0.0; rad = 0.0; rh = 0.0; alive = 0; }
          if (lane == 0) atomicAdd(&D.stat[C.d].merges, 1ull);
          // critical radii and contact thresholds follow the new body
          pair_consts();
        } else {
          const double R0q = SH(R0, q);
          fl = predicate_regs(xb_ - xa_, yb_ - ya_, zb_ - za_,
                              fma(zb_ - za_, zb_ - za_, fma(yb_ - ya_, yb_ - ya_, (xb_ - xa_) * (xb_ - xa_))),
                              vxb_ - vxa_, vyb_ - vya_, vzb_ - vza_, R0q * R0q * C.dp->ck2[k], h);
        }
      }
      if (lane == q) lev = fl ? k : k - 1;
      nonempty |= fl;
    }
    *merged = true;
    return nonempty;
  };

  int k = 1, deepest = 1, forces_at = -1;
  long long substeps = 0;
  hs[1] = C.dt / (double)C.M;
  cs[1] = 0;
  bool start = true, aborted = false;
  for (;;) {
    if (start) {
      // a single pair below this level: the packed single-pair path
      if (k >= 1 && C.l == 3) {
        const unsigned Lm = __ballot_sync(FULL, isp && lev >= k - 1);
        if (__popc(Lm) == 1) {
          const int q = __ffs(Lm) - 1;
          const int a_ = SH(ia, q), b_ = SH(ib, q);
          if (SH(alive, a_) && SH(alive, b_)) {
            const int pc = lane & 3, src = ((lane >> 2) & 1) ? b_ : a_;
            const double px = SH(x, src), py = SH(y, src), pz = SH(z, src);
            const double ux = SH(vx, src), uy = SH(vy, src), uz = SH(vz, src);
            double X = pc == 0 ? px : (pc == 1 ? py : (pc == 2 ? pz : 0.0));
            double V = pc == 0 ? ux : (pc == 1 ? uy : (pc == 2 ? uz : 0.0));
            int plev = SH(lev, q);
            const long long sub0 = substeps;
            const int rc = pair_run(D, C, lane, hs, cs, lc, X, V, SH(gm, a_), SH(gm, b_), SH(R0sq, q),
                                    SH(iR0, q), SH(Rcut, q), k, plev, substeps, deepest);
            if (lane == 0) atomicAdd(&D.stat[C.d].pair_substeps, (unsigned long long)(substeps - sub0));
            const double ax_ = SH(X, 0), ay_ = SH(X, 1), az_ = SH(X, 2);
            const double avx = SH(V, 0), avy = SH(V, 1), avz = SH(V, 2);
            const double bx_ = SH(X, 4), by_ = SH(X, 5), bz_ = SH(X, 6);
            const double bvx = SH(V, 4), bvy = SH(V, 5), bvz = SH(V, 6);
            if (lane == a_) { x = ax_; y = ay_; z = az_; vx = avx; vy = avy; vz = avz; }
            if (lane == b_) { x = bx_; y = by_; z = bz_; vx = bvx; vy = bvy; vz = bvz; }
            if (lane == q) lev = plev;
            forces_at = -1;
            if (rc == 0) {            // level k + 1 finished: continue with the closing kick of k
              if (k == 0) break;
              start = false;
              continue;
            }
            if (rc == 2) { aborted = true; break; }
            // rc == 1: a contact may be due; this sub-step takes the general path
          }
        }
      }
      ++substeps;
      if (substeps > C.max_substeps) { aborted = true; break; }
      deepest = max(deepest, k);
      bool merged = false;
      const bool fk = check(k, hs[k], &merged);
      if (merged || forces_at != k) { forces(k); forces_at = k; }
      kick(k, 0.5 * hs[k]);
      const bool deeper = fk && (k + 1 <= C.max_depth);
      if (fk && !deeper && lane == 0) set_status(&D.stat[C.d], SYMBA_E_DEPTH);
      drift(k, hs[k], fk && !deeper);
      if (deeper) {
        ++k;
        hs[k] = sub_interval(C, hs[k - 1]);
        cs[k] = 0;
        continue;
      }
      start = false;
    }
    forces(k);
    forces_at = k;
    kick(k, 0.5 * hs[k]);
    if (++cs[k] < C.M) { start = true; continue; }
    --k;
    forces_at = -1;
    if (k == 0) break;
  }
  if (aborted && lane == 0) set_status(&D.stat[C.d], SYMBA_E_DEPTH);
  if (lane == 0) {
    atomicMax(&D.stat[C.d].max_depth, deepest);
    atomicAdd(&D.stat[C.d].substeps, (unsigned long long)substeps);
    atomicMax(&D.stat[C.d].max_chain, (unsigned long long)substeps);
  }
  if (ism) {
    D.x[pglob] = x; D.y[pglob] = y; D.z[pglob] = z;
    D.vx[pglob] = vx; D.vy[pglob] = vy; D.vz[pglob] = vz;
    D.m[pglob] = m; D.gm[pglob] = gm; D.rad[pglob] = rad; D.rh[pglob] = rh;
    D.alive[pglob] = alive;
  }
  __syncwarp();
}

__device__ void run_group(const Dev &D, int g, int lane, const Levels &V, SmallView *sv, double *lc) {
  GroupCtx C;
  C.moff = D.g_moff[g];
  C.mcnt = D.g_mcnt[g];
  C.poff = D.g_poff[g];
  C.pcnt = D.g_pcnt[g];
  C.d = D.blk_disk[D.gmem[C.moff] >> 5];
  C.dp = &D.disks[C.d];
  C.M = C.dp->M; C.l = C.dp->l; C.max_depth = C.dp->max_depth; C.max_substeps = C.dp->max_substeps;
  C.dt = C.dp->dt; C.lam = C.dp->hill_scale; C.G = C.dp->G;
  C.mu = __dmul_rn(C.dp->G, C.dp->m0);
  C.invM = 1.0 / (double)C.M;

  if (C.mcnt <= 32 && C.pcnt <= 32) {
    run_group_regs(D, C, lane, V.h, V.cnt, lc);
    return;
  }
  GView S;
  const bool small = C.mcnt <= SMALL_M && C.pcnt <= SMALL_P;
  if (small) {
    S.x = sv->x; S.y = sv->y; S.z = sv->z; S.vx = sv->vx; S.vy = sv->vy; S.vz = sv->vz;
    S.m = sv->m; S.gm = sv->gm; S.rad = sv->rad; S.rh = sv->rh; S.alive = sv->alive;
    S.pa = sv->pa; S.pb = sv->pb; S.lev = sv->lev; S.R0 = sv->R0; S.invR0 = sv->invR0; S.pf = sv->pf;
    S.adj_off = sv->adj_off; S.adj_cnt = sv->adj_cnt; S.adj = sv->adj;
    S.perm = sv->perm; S.ptmp = sv->ptmp; S.mperm = sv->mperm; S.mtmp = sv->mtmp;
  } else {
    const size_t mo = C.moff, po = C.poff;
    S.x = D.gx + mo; S.y = D.gy + mo; S.z = D.gz + mo; S.vx = D.gvx + mo; S.vy = D.gvy + mo; S.vz = D.gvz + mo;
    S.m = D.gmm + mo; S.gm = D.ggm + mo; S.rad = D.grad + mo; S.rh = D.grh + mo; S.alive = D.galive + mo;
    S.pa = D.gpa + po; S.pb = D.gpb + po; S.lev = D.lev + po; S.R0 = D.pR0 + po; S.invR0 = D.pinvR0 + po;
    S.pf = D.pf + 5 * po;
    S.adj_off = D.adj_off + mo; S.adj_cnt = D.adj_cnt + mo; S.adj = D.adj + 2 * po;
    S.perm = D.perm + po; S.ptmp = D.ptmp + po; S.mperm = D.mperm + mo; S.mtmp = D.mtmp + mo;
  }

  // gather: member slots (ascending index), pairs as member-slot pairs, adjacency in pair order
  for (int a = lane; a < C.mcnt; a += 32) {
    const int p = D.gmem[C.moff + a];
    D.mslot[p] = a;
    S.x[a] = D.x[p]; S.y[a] = D.y[p]; S.z[a] = D.z[p];
    S.vx[a] = D.vx[p]; S.vy[a] = D.vy[p]; S.vz[a] = D.vz[p];
    S.m[a] = D.m[p]; S.gm[a] = D.gm[p]; S.rad[a] = D.rad[p]; S.rh[a] = D.rh[p];
    S.alive[a] = D.alive[p];
    S.adj_cnt[a] = 0;
    S.mperm[a] = a;
  }
  __syncwarp();
  for (int q = lane; q < C.pcnt; q += 32) {
    S.pa[q] = D.mslot[D.gpi[C.poff + q]];
    S.pb[q] = D.mslot[D.gpj[C.poff + q]];
    S.lev[q] = 0;
    S.perm[q] = q;
  }
  __syncwarp();
  for (int q = lane; q < C.pcnt; q += 32) set_r0(S, C, q);
  if (lane == 0) {
    int o = 0;
    for (int q = 0; q < C.pcnt; ++q) { S.adj_cnt[S.pa[q]]++; S.adj_cnt[S.pb[q]]++; }
    for (int a = 0; a < C.mcnt; ++a) { S.adj_off[a] = o; o += S.adj_cnt[a]; S.adj_cnt[a] = 0; }
    for (int q = 0; q < C.pcnt; ++q) {
      const int a = S.pa[q], b = S.pb[q];
      S.adj[S.adj_off[a] + S.adj_cnt[a]++] = q << 1;
      S.adj[S.adj_off[b] + S.adj_cnt[b]++] = (q << 1) | 1;
    }
  }
  __syncwarp();

  recurse(S, C, D, V, lane, lc);

  // scatter back
  for (int a = lane; a < C.mcnt; a += 32) {
    const int p = D.gmem[C.moff + a];
    D.x[p] = S.x[a]; D.y[p] = S.y[a]; D.z[p] = S.z[a];
    D.vx[p] = S.vx[a]; D.vy[p] = S.vy[a]; D.vz[p] = S.vz[a];
    D.m[p] = S.m[a]; D.gm[p] = S.gm[a]; D.rad[p] = S.rad[a]; D.rh[p] = S.rh[a];
    D.alive[p] = S.alive[a];
  }
  __syncwarp();
}

__global__ void __launch_bounds__(128) k_recursion(Dev D) {
  __shared__ double hs[4][SYM_MAX_LEVELS + 2];
  __shared__ int cs[4][SYM_MAX_LEVELS + 2], ls[4][SYM_MAX_LEVELS + 2], ms[4][SYM_MAX_LEVELS + 2];
  __shared__ SmallView sview[4];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const Levels V{hs[w], cs[w], ls[w], ms[w]};
  double *lc = D.lcache + (size_t)(blockIdx.x * 4 + w) * SYM_PAIR_LC;
  const int total = *D.rec_total;
  for (;;) {
    int item = 0;
    if (lane == 0) item = atomicAdd(&D.work[2], 1);
    item = __shfl_sync(FULL, item, 0);
    if (item >= total) break;
    run_group(D, D.rec_items[item], lane, V, &sview[w], lc);
  }
}

int recursion_blocks_per_sm() { return 1; }

void launch_recursion(const Dev &D, const LaunchCfg &L, cudaStream_t s) {
  k_recursion<<<L.rec_blocks, 128, 0, s>>>(D);
}
