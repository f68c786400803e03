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
// quadrant), so the path is kept short: the deep-level drift uses the Lagrange f and g series
// when the sub-step is a tiny fraction of the orbit, square roots come from an integer-built FP32
// seed plus one FP64 correction, the shell weights use per-level reciprocal tables, and the
// forces of the closing kick of one sub-step are reused by the opening kick of the next (same
// positions, same pairs, same weights).  The check below level 0 uses the division-free form of
// the predicate (same minimum-distance test; identical except at exact ties).
#include "internal.cuh"

#define FULL 0xffffffffu

struct GroupCtx {
  int d, moff, mcnt, poff, pcnt;
  int M, l, max_depth, max_substeps;
  double dt, lam, G, mu;
  const DiskDesc *dp;
};

// exact contact test: |x_j - x_i|^2 < (R_i + R_j)^2, one IEEE operation at a time
__device__ __forceinline__ bool contact(const Dev &D, int i, int j) {
  const double dx = __dsub_rn(D.x[j], D.x[i]), dy = __dsub_rn(D.y[j], D.y[i]), dz = __dsub_rn(D.z[j], D.z[i]);
  const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
  const double Rc = __dadd_rn(D.rad[i], D.rad[j]);
  return r2 < __dmul_rn(Rc, Rc);
}

// minimum distance of the straight-line relative motion over [0, h] below R_k (division-free)
__device__ __forceinline__ bool predicate_fast(const Dev &D, int i, int j, double R2, double h) {
  const double dx = D.x[j] - D.x[i], dy = D.y[j] - D.y[i], dz = D.z[j] - D.z[i];
  const double dvx = D.vx[j] - D.vx[i], dvy = D.vy[j] - D.vy[i], dvz = D.vz[j] - D.vz[i];
  const double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
  if (r2 < R2) return true;
  const double vr = fma(dz, dvz, fma(dy, dvy, dx * dvx));
  if (vr >= 0.0) return false;
  const double v2 = fma(dvz, dvz, fma(dvy, dvy, dvx * dvx));
  if (-vr < h * v2) return fma(r2, v2, -vr * vr) < R2 * v2;
  return fma(h, fma(h, v2, 2.0 * vr), r2) < R2;
}

__device__ __forceinline__ void set_r0(const Dev &D, const GroupCtx &C, int q) {
  const int i = D.gpi[q], j = D.gpj[q];
  const double R0 = __dmul_rn(C.lam, __dadd_rn(D.rh[i], D.rh[j]));
  D.pR0[q] = R0;
  D.pinvR0[q] = R0 > 0.0 ? 1.0 / R0 : 0.0;
}

// merger of j into i (i < j): summed mass, mass-weighted position and barycentric velocity,
// radius (R_i^3 + R_j^3)^{1/3}, Hill radius rH_i (m / m_i)^{1/3}; j leaves the system.
__device__ void merge_pair(const Dev &D, const GroupCtx &C, int i, int j) {
  const double mi = D.m[i], mj = D.m[j];
  const double M = __dadd_rn(mi, mj);
  if (M > 0.0) {
    D.x[i] = __ddiv_rn(__dadd_rn(__dmul_rn(mi, D.x[i]), __dmul_rn(mj, D.x[j])), M);
    D.y[i] = __ddiv_rn(__dadd_rn(__dmul_rn(mi, D.y[i]), __dmul_rn(mj, D.y[j])), M);
    D.z[i] = __ddiv_rn(__dadd_rn(__dmul_rn(mi, D.z[i]), __dmul_rn(mj, D.z[j])), M);
    D.vx[i] = __ddiv_rn(__dadd_rn(__dmul_rn(mi, D.vx[i]), __dmul_rn(mj, D.vx[j])), M);
    D.vy[i] = __ddiv_rn(__dadd_rn(__dmul_rn(mi, D.vy[i]), __dmul_rn(mj, D.vy[j])), M);
    D.vz[i] = __ddiv_rn(__dadd_rn(__dmul_rn(mi, D.vz[i]), __dmul_rn(mj, D.vz[j])), M);
  }
  const double Ri = D.rad[i], Rj = D.rad[j];
  D.rad[i] = cbrt(__dadd_rn(__dmul_rn(__dmul_rn(Ri, Ri), Ri), __dmul_rn(__dmul_rn(Rj, Rj), Rj)));
  if (mi > 0.0) D.rh[i] = __dmul_rn(D.rh[i], cbrt(__ddiv_rn(M, mi)));
  D.m[i] = M;
  D.gm[i] = __dmul_rn(C.G, M);
  D.m[j] = 0.0;
  D.gm[j] = 0.0;
  D.rad[j] = 0.0;
  D.rh[j] = 0.0;
  D.alive[j] = 0;
  atomicAdd(&D.stat[C.d].merges, 1ull);
  // the critical radii of i's pairs change with its Hill radius
  const int a = D.mslot[i];
  const int ao = D.adj_off[C.moff + a], ac = D.adj_cnt[C.moff + a];
  for (int e = 0; e < ac; ++e) set_r0(D, C, C.poff + (D.adj[2 * (size_t)C.poff + ao + e] >> 1));
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

// (i): level-k check of F_{k-1} (= the first lenL[k] entries of perm).  Returns whether F_k is
// non-empty; sets *merged when bodies merged.
__device__ bool check_level(const Dev &D, const GroupCtx &C, const Levels &V, int k, int lane,
                            bool *merged) {
  int *lev = D.lev + C.poff;
  const int *perm = D.perm + C.poff;
  const int L = V.lenL[k];
  const double h = V.h[k];
  bool any_contact = false;
  for (int b = 0; b < L; b += 32) {
    const int t = b + lane;
    bool ct = false;
    if (t < L) {
      const int q = C.poff + perm[t];
      const int i = D.gpi[q], j = D.gpj[q];
      if (D.alive[i] && D.alive[j]) ct = contact(D, i, j);
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
        const int ql = perm[t], q = C.poff + ql;
        const int i = D.gpi[q], j = D.gpj[q];
        if (D.alive[i] && D.alive[j]) {
          const double R0 = D.pR0[q];
          fl = predicate_fast(D, i, j, R0 * R0 * ck2, h);
        }
        lev[ql] = fl ? k : k - 1;
      }
      nonempty |= (__any_sync(FULL, fl) != 0);
    }
    *merged = false;
  } else {
    // a merger changes bodies that later pairs read: take the pairs one by one in list order
    if (lane == 0) {
      for (int ql = 0; ql < C.pcnt; ++ql) {
        if (lev[ql] < k - 1) continue;
        const int q = C.poff + ql;
        const int i = D.gpi[q], j = D.gpj[q];
        bool fl = false;
        if (D.alive[i] && D.alive[j]) {
          if (contact(D, i, j)) merge_pair(D, C, i, j);
          else {
            const double R0 = D.pR0[q];
            fl = predicate_fast(D, i, j, R0 * R0 * ck2, h);
          }
        }
        lev[ql] = fl ? k : k - 1;
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
__device__ void forces_level(const Dev &D, const GroupCtx &C, const Levels &V, int k, int lane) {
  const int *perm = D.perm + C.poff;
  double *pf = D.pf + 5 * (size_t)C.poff;
  const int L = V.lenL[k];
  const double ck = C.dp->ck[k], ck1 = C.dp->ck[k + 1], idk = C.dp->invdc[k];
  const double idkm = k > 0 ? C.dp->invdc[k - 1] : 0.0;
  for (int t = lane; t < L; t += 32) {
    const int ql = perm[t], q = C.poff + ql;
    const int i = D.gpi[q], j = D.gpj[q];
    double fi = 0.0, fj = 0.0, dx = 0.0, dy = 0.0, dz = 0.0;
    if (D.alive[i] && D.alive[j]) {
      dx = D.x[j] - D.x[i];
      dy = D.y[j] - D.y[i];
      dz = D.z[j] - D.z[i];
      const double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
      const double ri = rsqrt_fp64(r2);
      const double rho = r2 * ri * D.pinvR0[q];     // r / R_0
      double w = partition_fn((rho - ck1) * idk, C.l);
      if (k > 0) w -= partition_fn((rho - ck) * idkm, C.l);
      const double s = w * (ri * ri * ri);
      fi = D.gm[j] * s;
      fj = D.gm[i] * s;
    }
    pf[5 * ql + 0] = dx; pf[5 * ql + 1] = dy; pf[5 * ql + 2] = dz;
    pf[5 * ql + 3] = fi; pf[5 * ql + 4] = fj;
  }
  __syncwarp();
}

// kick hh of the bodies of F_{k-1} (the first lenM[k] member slots of mperm) with the forces in pf
__device__ void kick_level(const Dev &D, const GroupCtx &C, const Levels &V, int k, double hh, int lane) {
  const int *lev = D.lev + C.poff;
  const int *mperm = D.mperm + C.moff;
  const double *pf = D.pf + 5 * (size_t)C.poff;
  const int L = V.lenM[k];
  for (int t = lane; t < L; t += 32) {
    const int a = mperm[t];
    const int p = D.gmem[C.moff + a];
    if (!D.alive[p]) continue;
    const int ao = D.adj_off[C.moff + a], ac = D.adj_cnt[C.moff + a];
    double ax = 0.0, ay = 0.0, az = 0.0;
    for (int e = 0; e < ac; ++e) {
      const int code = D.adj[2 * (size_t)C.poff + ao + e];
      const int ql = code >> 1;
      if (lev[ql] < k - 1) continue;
      const double *f = pf + 5 * ql;
      if ((code & 1) == 0) { ax = fma(f[3], f[0], ax); ay = fma(f[3], f[1], ay); az = fma(f[3], f[2], az); }
      else { ax = fma(-f[4], f[0], ax); ay = fma(-f[4], f[1], ay); az = fma(-f[4], f[2], az); }
    }
    D.vx[p] = fma(hh, ax, D.vx[p]);
    D.vy[p] = fma(hh, ay, D.vy[p]);
    D.vz[p] = fma(hh, az, D.vz[p]);
  }
  __syncwarp();
}

// (iii): drift h the bodies of mperm[from..to)
__device__ void drift_range(const Dev &D, const GroupCtx &C, int from, int to, double h, int lane) {
  const int *mperm = D.mperm + C.moff;
  for (int t = from + lane; t < to; t += 32) {
    const int p = D.gmem[C.moff + mperm[t]];
    if (!D.alive[p]) continue;
    double x = D.x[p], y = D.y[p], z = D.z[p], vx = D.vx[p], vy = D.vy[p], vz = D.vz[p];
    if (!drift_series(C.mu, h, x, y, z, vx, vy, vz)) {
      const int st = kepler_drift(C.mu, h, x, y, z, vx, vy, vz);
      if (st != SYMBA_OK) set_status(&D.stat[C.d], st);
    }
    D.x[p] = x; D.y[p] = y; D.z[p] = z;
    D.vx[p] = vx; D.vy[p] = vy; D.vz[p] = vz;
  }
  __syncwarp();
}

__device__ void run_group(const Dev &D, int g, int lane, const Levels &V) {
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

  // member slots, pair adjacency in pair-list order, critical radii, initial lists
  for (int a = lane; a < C.mcnt; a += 32) {
    D.mslot[D.gmem[C.moff + a]] = a;
    D.adj_cnt[C.moff + a] = 0;
    D.mperm[C.moff + a] = a;
  }
  for (int ql = lane; ql < C.pcnt; ql += 32) {
    D.lev[C.poff + ql] = 0;
    D.perm[C.poff + ql] = ql;
  }
  __syncwarp();
  for (int ql = lane; ql < C.pcnt; ql += 32) set_r0(D, C, C.poff + ql);
  if (lane == 0) {
    int o = 0;
    for (int ql = 0; ql < C.pcnt; ++ql) {
      D.adj_cnt[C.moff + D.mslot[D.gpi[C.poff + ql]]]++;
      D.adj_cnt[C.moff + D.mslot[D.gpj[C.poff + ql]]]++;
    }
    for (int a = 0; a < C.mcnt; ++a) {
      D.adj_off[C.moff + a] = o;
      o += D.adj_cnt[C.moff + a];
      D.adj_cnt[C.moff + a] = 0;
    }
    for (int ql = 0; ql < C.pcnt; ++ql) {
      const int ai = D.mslot[D.gpi[C.poff + ql]], aj = D.mslot[D.gpj[C.poff + ql]];
      D.adj[2 * (size_t)C.poff + D.adj_off[C.moff + ai] + D.adj_cnt[C.moff + ai]++] = ql << 1;
      D.adj[2 * (size_t)C.poff + D.adj_off[C.moff + aj] + D.adj_cnt[C.moff + aj]++] = (ql << 1) | 1;
    }
  }
  __syncwarp();

  const int *lev = D.lev + C.poff;
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
      const bool fk = check_level(D, C, V, k, lane, &merged);
      if (merged || forces_at != k) { forces_level(D, C, V, k, lane); forces_at = k; }
      kick_level(D, C, V, k, 0.5 * V.h[k], lane);
      const bool deeper = fk && (k + 1 <= C.max_depth);
      if (fk && !deeper && lane == 0) set_status(&D.stat[C.d], SYMBA_E_DEPTH);
      int lm1 = 0;
      if (deeper) {
        // F_k and its bodies become the prefixes of the next level
        const int lp = partition_prefix(D.perm + C.poff, D.ptmp + C.poff, V.lenL[k],
                                        [&](int ql) { return lev[ql] == k; }, lane);
        lm1 = partition_prefix(D.mperm + C.moff, D.mtmp + C.moff, V.lenM[k],
                               [&](int a) {
                                 const int ao = D.adj_off[C.moff + a], ac = D.adj_cnt[C.moff + a];
                                 for (int e = 0; e < ac; ++e)
                                   if (lev[D.adj[2 * (size_t)C.poff + ao + e] >> 1] >= k) return true;
                                 return false;
                               }, lane);
        V.lenL[k + 1] = lp;
        V.lenM[k + 1] = lm1;
      }
      drift_range(D, C, lm1, V.lenM[k], V.h[k], lane);
      if (deeper) {
        ++k;
        V.h[k] = V.h[k - 1] / (double)C.M;
        V.cnt[k] = 0;
        continue;
      }
      start = false;
    }
    // (iv) of E_k, then the next of its M calls or back to the parent's (iv)
    forces_level(D, C, V, k, lane);
    forces_at = k;
    kick_level(D, C, V, k, 0.5 * V.h[k], lane);
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

__global__ void __launch_bounds__(128) k_recursion(Dev D) {
  __shared__ double hs[4][SYM_MAX_LEVELS + 2];
  __shared__ int cs[4][SYM_MAX_LEVELS + 2], ls[4][SYM_MAX_LEVELS + 2], ms[4][SYM_MAX_LEVELS + 2];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const Levels V{hs[w], cs[w], ls[w], ms[w]};
  const int total = *D.rec_total;
  for (;;) {
    int item = 0;
    if (lane == 0) item = atomicAdd(&D.work[2], 1);
    item = __shfl_sync(FULL, item, 0);
    if (item >= total) break;
    run_group(D, D.rec_items[item], lane, V);
  }
}

int recursion_blocks_per_sm() { return 1; }

void launch_recursion(const Dev &D, const LaunchCfg &L, cudaStream_t s) {
  k_recursion<<<L.rec_blocks, 128, 0, s>>>(D);
}
