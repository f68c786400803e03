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
// The sub-step chain is latency-bound (GB300 issues one FP64 warp instruction per ~64 cycles per
// quadrant), so it is kept short:
//   - the group's bodies and pairs are gathered into a member-slot view that lives in shared
//     memory for groups of up to 32 bodies and 64 pairs (global scratch otherwise), so phases
//     exchange data through shared memory, and are scattered back at the end;
//   - the deep-level drift uses the Lagrange f and g series when the sub-step is a tiny fraction
//     of the orbit; square roots come from an integer-built FP32 seed plus one FP64 correction;
//     the shell weights use per-level reciprocal tables;
//   - the forces of the closing kick of one sub-step are reused by the opening kick of the next
//     (same positions, same pairs, same weights).
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
  double dt, lam, G, mu;
  const DiskDesc *dp;
};

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
  S.rad[a] = cbrt(__dadd_rn(__dmul_rn(__dmul_rn(Ra, Ra), Ra), __dmul_rn(__dmul_rn(Rb, Rb), Rb)));
  if (ma > 0.0) S.rh[a] = __dmul_rn(S.rh[a], cbrt(__ddiv_rn(M, ma)));
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

__device__ void recurse(const GView &S, const GroupCtx &C, const Dev &D, const Levels &V, int lane) {
  int k = 1, deepest = 1, forces_at = -1;
  long long substeps = 0;
  V.h[1] = C.dt / (double)C.M;
  V.cnt[1] = 0;
  V.lenL[1] = C.pcnt;
  V.lenM[1] = C.mcnt;
  bool start = true, aborted = false;
  for (;;) {
    if (start) {
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
        V.h[k] = V.h[k - 1] / (double)C.M;
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

__device__ void run_group_regs(const Dev &D, const GroupCtx &C, int lane, double *hs, int *cs) {
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
            rad = cbrt(__dadd_rn(__dmul_rn(__dmul_rn(ra_, ra_), ra_), __dmul_rn(__dmul_rn(rb_, rb_), rb_)));
            if (ma > 0.0) rh = __dmul_rn(rha, cbrt(__ddiv_rn(Mt, ma)));
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
        hs[k] = hs[k - 1] / (double)C.M;
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
  }
  if (ism) {
    D.x[pglob] = x; D.y[pglob] = y; D.z[pglob] = z;
    D.vx[pglob] = vx; D.vy[pglob] = vy; D.vz[pglob] = vz;
    D.m[pglob] = m; D.gm[pglob] = gm; D.rad[pglob] = rad; D.rh[pglob] = rh;
    D.alive[pglob] = alive;
  }
  __syncwarp();
}

__device__ void run_group(const Dev &D, int g, int lane, const Levels &V, SmallView *sv) {
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

  if (C.mcnt <= 32 && C.pcnt <= 32) {
    run_group_regs(D, C, lane, V.h, V.cnt);
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

  recurse(S, C, D, V, lane);

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
  const int total = *D.rec_total;
  for (;;) {
    int item = 0;
    if (lane == 0) item = atomicAdd(&D.work[2], 1);
    item = __shfl_sync(FULL, item, 0);
    if (item >= total) break;
    run_group(D, D.rec_items[item], lane, V, &sview[w]);
  }
}

int recursion_blocks_per_sm() { return 1; }

void launch_recursion(const Dev &D, const LaunchCfg &L, cudaStream_t s) {
  k_recursion<<<L.rec_blocks, 128, 0, s>>>(D);
}
