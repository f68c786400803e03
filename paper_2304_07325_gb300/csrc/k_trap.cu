// The right-angled-trapezoid pair kick (Sec. 2): every pair i < N_m, j > i once, both
// reactions accumulated, no atomics.
//
// Work decomposition.  Indices are cut into 32-blocks; tile (I, J), I <= J, I < ceil(N_m/32),
// holds the pairs of block I (rows) with block J (columns): the trapezoid becomes a rectangle of
// off-diagonal tiles plus the diagonal tiles of the triangle, all in one flat list that
// persistent warps consume in segments from a counter (the fold of the triangle into a
// rectangle, done by a work queue instead of index arithmetic).
//
// One warp per tile.  Lane l keeps row particle I*32+l in registers; the column particles
// rotate through the lanes with warp shuffles (32 steps; 16 on a diagonal tile, where each
// unordered pair is met once), each carrying its own accumulator, so after the sweep every
// column accumulator is back in its home lane.  Both sides are written as per-tile partials
// and summed later in a fixed order: the result does not depend on scheduling, segment length
// or which other systems share the launch.
//
// FP64 path: 16 FP64-pipe instructions per pair (3 differences, 3 for r^2, 2 for r^-3 -- its seed,
// Newton step and powers run on the integer pipe -- 2 mass scalings, 6 FMAs into the two
// accumulators).
//
// Kick 1 also runs the close-encounter check (Sec. 2) of every pair: a conservative FP32
// prefilter (|d| - tau |dv| against R_0 with rounding margins) and, for the rare pairs that pass,
// the exact FP64 predicate, identical operation for operation to the definition; flagged pairs
// are appended to the system's pair list and weighted by g_0(r).  Kick 2 weights the same
// flagged pairs, found through the group each particle belongs to.
#include "internal.cuh"

#define FULL 0xffffffffu

struct TileCtx {
  int off, n, nm, pair_base, pair_cap, l;
  double dt, lam, c0, c1;
};

__device__ __forceinline__ TileCtx load_ctx(const DiskDesc *dp) {
  TileCtx c;
  c.off = dp->off; c.n = dp->n; c.nm = dp->nm;
  c.pair_base = dp->pair_base; c.pair_cap = dp->pair_cap; c.l = dp->l;
  c.dt = dp->dt; c.lam = dp->hill_scale; c.c0 = dp->ck[0]; c.c1 = dp->ck[1];
  return c;
}

__device__ __forceinline__ double g0_weight(const TileCtx &c, double R0, double r) {
  const double Rk = R0 * c.c0, Rk1 = R0 * c.c1;
  return partition_fn((r - Rk1) / (Rk - Rk1), c.l);
}

// Binary search of (lo, hi) in the sorted pair list of a group.
__device__ __forceinline__ bool group_has_pair(const Dev &D, int g, int lo, int hi) {
  int a = D.g_poff[g], b = a + D.g_pcnt[g];
  while (a < b) {
    const int m = (a + b) >> 1;
    const int mi = D.gpi[m], mj = D.gpj[m];
    if (mi < lo || (mi == lo && mj < hi)) a = m + 1; else b = m;
  }
  return a < D.g_poff[g] + D.g_pcnt[g] && D.gpi[a] == lo && D.gpj[a] == hi;
}

template <int MODE>
__device__ __forceinline__ void tile_fp64(const Dev &D, const TileCtx &c, const DiskDesc *dp,
                                          int t, int4 tl, int lane) {
  const bool diag = tl.y == tl.z;
  const int pi = tl.y * 32 + lane;
  const int li = pi - c.off;
  const bool live_i = li < c.n && D.alive[pi];
  const bool row_i = live_i && li < c.nm;
  const double xi = D.x[pi], yi = D.y[pi], zi = D.z[pi], gmi = D.gm[pi];
  double axi = 0.0, ayi = 0.0, azi = 0.0;

  int jid = tl.z * 32 + lane;
  const int lj0 = jid - c.off;
  const bool live_j0 = lj0 < c.n && D.alive[jid];
  int jflags = (live_j0 ? 1 : 0) | ((live_j0 && lj0 < c.nm) ? 2 : 0);
  double xj = D.x[jid], yj = D.y[jid], zj = D.z[jid], gmj = D.gm[jid];
  double axj = 0.0, ayj = 0.0, azj = 0.0;

  // kick 1: FP32 prefilter data; kick 2: group ids
  float xfi = 0.f, yfi = 0.f, zfi = 0.f, vxfi = 0.f, vyfi = 0.f, vzfi = 0.f, lami = 0.f, sigi = 0.f;
  float xfj = 0.f, yfj = 0.f, zfj = 0.f, vxfj = 0.f, vyfj = 0.f, vzfj = 0.f, lamj = 0.f, sigj = 0.f;
  int gidi = -1, gidj = -1;
  if (MODE == 1) {
    xfi = D.xf[pi]; yfi = D.yf[pi]; zfi = D.zf[pi];
    vxfi = D.vxf[pi]; vyfi = D.vyf[pi]; vzfi = D.vzf[pi];
    lami = D.lamf[pi]; sigi = D.sigf[pi];
    xfj = D.xf[jid]; yfj = D.yf[jid]; zfj = D.zf[jid];
    vxfj = D.vxf[jid]; vyfj = D.vyf[jid]; vzfj = D.vzf[jid];
    lamj = D.lamf[jid]; sigj = D.sigf[jid];
  } else {
    gidi = D.gid[pi];
    gidj = D.gid[jid];
  }
  const float tauf = __double2float_ru(c.dt);

  auto rotate = [&]() {
    const int src = (lane + 1) & 31;
    xj = __shfl_sync(FULL, xj, src); yj = __shfl_sync(FULL, yj, src);
    zj = __shfl_sync(FULL, zj, src); gmj = __shfl_sync(FULL, gmj, src);
    axj = __shfl_sync(FULL, axj, src); ayj = __shfl_sync(FULL, ayj, src);
    azj = __shfl_sync(FULL, azj, src);
    jid = __shfl_sync(FULL, jid, src); jflags = __shfl_sync(FULL, jflags, src);
    if (MODE == 1) {
      xfj = __shfl_sync(FULL, xfj, src); yfj = __shfl_sync(FULL, yfj, src);
      zfj = __shfl_sync(FULL, zfj, src); vxfj = __shfl_sync(FULL, vxfj, src);
      vyfj = __shfl_sync(FULL, vyfj, src); vzfj = __shfl_sync(FULL, vzfj, src);
      lamj = __shfl_sync(FULL, lamj, src); sigj = __shfl_sync(FULL, sigj, src);
    } else {
      gidj = __shfl_sync(FULL, gidj, src);
    }
  };

  const int nsteps = diag ? 16 : 32;
  if (diag) rotate();
#pragma unroll 1
  for (int s = 0; s < nsteps; ++s) {
    bool valid;
    if (!diag) {
      valid = row_i && (jflags & 1);
    } else {
      valid = (jid > pi) ? (row_i && (jflags & 1)) : (live_i && (jflags & 2));
      if (s == 15 && lane >= 16) valid = false;  // pair {l, l+16} belongs to lane l < 16
    }
    const double dx = xj - xi, dy = yj - yi, dz = zj - zi;
    const double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
    const double r3 = rinv3(r2);
    double sj = gmj * r3;
    double si = gmi * r3;
    if (MODE == 1) {
      const float dxf = xfj - xfi, dyf = yfj - yfi, dzf = zfj - zfi;
      const float r2f = fmaf(dzf, dzf, fmaf(dyf, dyf, dxf * dxf));
      const float dvxf = vxfj - vxfi, dvyf = vyfj - vyfi, dvzf = vzfj - vzfi;
      const float vmag = sqrtf(fmaf(dvzf, dvzf, fmaf(dvyf, dvyf, dvxf * dvxf)));
      const float Bf = fmaf(tauf, vmag, lami + lamj) * 1.0000039f + 1.9073486e-6f * (sigi + sigj);
      const bool cand = valid && !(r2f > Bf * Bf);
      if (__any_sync(FULL, cand)) {
        if (cand) {
          const int lo = min(pi, jid), hi = max(pi, jid);
          const double ex = __dsub_rn(D.x[hi], D.x[lo]), ey = __dsub_rn(D.y[hi], D.y[lo]),
                       ez = __dsub_rn(D.z[hi], D.z[lo]);
          const double evx = __dsub_rn(D.vx[hi], D.vx[lo]), evy = __dsub_rn(D.vy[hi], D.vy[lo]),
                       evz = __dsub_rn(D.vz[hi], D.vz[lo]);
          const double R0 = __dmul_rn(c.lam, __dadd_rn(D.rh[lo], D.rh[hi]));
          if (encounter_exact(ex, ey, ez, evx, evy, evz, R0, c.dt)) {
            const int k = atomicAdd(&D.stat[tl.x].npairs, 1);
            if (k < c.pair_cap) {
              D.raw_i[c.pair_base + k] = lo;
              D.raw_j[c.pair_base + k] = hi;
            }
            const double er2 = __dadd_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)), __dmul_rn(ez, ez));
            const double w = g0_weight(c, R0, __dsqrt_rn(er2));
            sj *= w;
            si *= w;
          }
        }
      }
    } else {
      if (gidi >= 0 && gidi == gidj && valid) {
        const int lo = min(pi, jid), hi = max(pi, jid);
        if (group_has_pair(D, gidi, lo, hi)) {
          const double R0 = __dmul_rn(c.lam, __dadd_rn(D.rh[lo], D.rh[hi]));
          const double w = g0_weight(c, R0, sqrt(r2));
          sj *= w;
          si *= w;
        }
      }
    }
    sj = keep_or_zero(sj, valid);
    si = keep_or_zero(si, valid);
    axi = fma(sj, dx, axi); ayi = fma(sj, dy, ayi); azi = fma(sj, dz, azi);
    axj = fma(-si, dx, axj); ayj = fma(-si, dy, ayj); azj = fma(-si, dz, azj);
    if (!diag || s + 1 < nsteps) rotate();
  }
  (void)dp;
  double *out = D.part + (size_t)t * 2 * 3 * 32 + lane;
  if (diag) {
    const int src = (lane + 16) & 31;
    axi += __shfl_sync(FULL, axj, src);
    ayi += __shfl_sync(FULL, ayj, src);
    azi += __shfl_sync(FULL, azj, src);
    out[0] = axi; out[32] = ayi; out[64] = azi;
  } else {
    out[0] = axi; out[32] = ayi; out[64] = azi;
    out[96] = axj; out[128] = ayj; out[160] = azj;
  }
}

// Mixed precision (FP32 pair path): the relative displacement is formed from the two-float split
// x = xf + xl of each FP64 position, (xf_j - xf_i) + (xl_j - xl_i), which is exact in the high
// part for nearby bodies and within one FP32 ulp of the rounded FP64 difference otherwise; r^-3
// from the FP32 rsqrt plus one Newton step; both sides accumulated in FP32 with Kahan
// compensation and written as (sum, compensation) pairs that the reduction carries into FP64.
// The encounter check is the same FP64 decision as in the FP64 path.
__device__ __forceinline__ void kahan(float &s, float &c, float term) {
  const float y = term - c;
  const float t = s + y;
  c = (t - s) - y;
  s = t;
}

template <int MODE>
__device__ __forceinline__ void tile_mixed(const Dev &D, const TileCtx &c, int t, int4 tl, int lane) {
  const bool diag = tl.y == tl.z;
  const int pi = tl.y * 32 + lane;
  const int li = pi - c.off;
  const bool live_i = li < c.n && D.alive[pi];
  const bool row_i = live_i && li < c.nm;
  const float xhi = D.xf[pi], yhi = D.yf[pi], zhi = D.zf[pi];
  const float xlo = D.xl[pi], ylo = D.yl[pi], zlo = D.zl[pi];
  const float gmi = D.gmf[pi];
  float sxi = 0.f, syi = 0.f, szi = 0.f, cxi = 0.f, cyi = 0.f, czi = 0.f;

  int jid = tl.z * 32 + lane;
  const int lj0 = jid - c.off;
  const bool live_j0 = lj0 < c.n && D.alive[jid];
  int jflags = (live_j0 ? 1 : 0) | ((live_j0 && lj0 < c.nm) ? 2 : 0);
  float xhj = D.xf[jid], yhj = D.yf[jid], zhj = D.zf[jid];
  float xlj = D.xl[jid], ylj = D.yl[jid], zlj = D.zl[jid];
  float gmj = D.gmf[jid];
  float sxj = 0.f, syj = 0.f, szj = 0.f, cxj = 0.f, cyj = 0.f, czj = 0.f;

  float vxfi = 0.f, vyfi = 0.f, vzfi = 0.f, lami = 0.f, sigi = 0.f;
  float vxfj = 0.f, vyfj = 0.f, vzfj = 0.f, lamj = 0.f, sigj = 0.f;
  int gidi = -1, gidj = -1;
  if (MODE == 1) {
    vxfi = D.vxf[pi]; vyfi = D.vyf[pi]; vzfi = D.vzf[pi]; lami = D.lamf[pi]; sigi = D.sigf[pi];
    vxfj = D.vxf[jid]; vyfj = D.vyf[jid]; vzfj = D.vzf[jid]; lamj = D.lamf[jid]; sigj = D.sigf[jid];
  } else {
    gidi = D.gid[pi];
    gidj = D.gid[jid];
  }
  const float tauf = __double2float_ru(c.dt);

  auto rotate = [&]() {
    const int src = (lane + 1) & 31;
    xhj = __shfl_sync(FULL, xhj, src); yhj = __shfl_sync(FULL, yhj, src); zhj = __shfl_sync(FULL, zhj, src);
    xlj = __shfl_sync(FULL, xlj, src); ylj = __shfl_sync(FULL, ylj, src); zlj = __shfl_sync(FULL, zlj, src);
    gmj = __shfl_sync(FULL, gmj, src);
    sxj = __shfl_sync(FULL, sxj, src); syj = __shfl_sync(FULL, syj, src); szj = __shfl_sync(FULL, szj, src);
    cxj = __shfl_sync(FULL, cxj, src); cyj = __shfl_sync(FULL, cyj, src); czj = __shfl_sync(FULL, czj, src);
    jid = __shfl_sync(FULL, jid, src); jflags = __shfl_sync(FULL, jflags, src);
    if (MODE == 1) {
      vxfj = __shfl_sync(FULL, vxfj, src); vyfj = __shfl_sync(FULL, vyfj, src);
      vzfj = __shfl_sync(FULL, vzfj, src); lamj = __shfl_sync(FULL, lamj, src);
      sigj = __shfl_sync(FULL, sigj, src);
    } else {
      gidj = __shfl_sync(FULL, gidj, src);
    }
  };

  const int nsteps = diag ? 16 : 32;
  if (diag) rotate();
#pragma unroll 1
  for (int s = 0; s < nsteps; ++s) {
    bool valid;
    if (!diag) {
      valid = row_i && (jflags & 1);
    } else {
      valid = (jid > pi) ? (row_i && (jflags & 1)) : (live_i && (jflags & 2));
      if (s == 15 && lane >= 16) valid = false;
    }
    const float dx = (xhj - xhi) + (xlj - xlo);
    const float dy = (yhj - yhi) + (ylj - ylo);
    const float dz = (zhj - zhi) + (zlj - zlo);
    const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
    float ri;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(ri) : "f"(r2));
    ri = ri * fmaf(-0.5f * r2, ri * ri, 1.5f);
    const float s3 = ri * ri * ri;
    float sj = gmj * s3, si = gmi * s3;
    if (MODE == 1) {
      const float dvxf = vxfj - vxfi, dvyf = vyfj - vyfi, dvzf = vzfj - vzfi;
      const float vmag = sqrtf(fmaf(dvzf, dvzf, fmaf(dvyf, dvyf, dvxf * dvxf)));
      const float Bf = fmaf(tauf, vmag, lami + lamj) * 1.0000039f + 1.9073486e-6f * (sigi + sigj);
      const bool cand = valid && !(r2 > Bf * Bf * 1.0000153f);
      if (__any_sync(FULL, cand)) {
        if (cand) {
          const int lo = min(pi, jid), hi = max(pi, jid);
          const double ex = __dsub_rn(D.x[hi], D.x[lo]), ey = __dsub_rn(D.y[hi], D.y[lo]),
                       ez = __dsub_rn(D.z[hi], D.z[lo]);
          const double evx = __dsub_rn(D.vx[hi], D.vx[lo]), evy = __dsub_rn(D.vy[hi], D.vy[lo]),
                       evz = __dsub_rn(D.vz[hi], D.vz[lo]);
          const double R0 = __dmul_rn(c.lam, __dadd_rn(D.rh[lo], D.rh[hi]));
          if (encounter_exact(ex, ey, ez, evx, evy, evz, R0, c.dt)) {
            const int k = atomicAdd(&D.stat[tl.x].npairs, 1);
            if (k < c.pair_cap) {
              D.raw_i[c.pair_base + k] = lo;
              D.raw_j[c.pair_base + k] = hi;
            }
            const double er2 = __dadd_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)), __dmul_rn(ez, ez));
            const float w = (float)g0_weight(c, R0, __dsqrt_rn(er2));
            sj *= w;
            si *= w;
          }
        }
      }
    } else {
      if (gidi >= 0 && gidi == gidj && valid) {
        const int lo = min(pi, jid), hi = max(pi, jid);
        if (group_has_pair(D, gidi, lo, hi)) {
          const double R0 = __dmul_rn(c.lam, __dadd_rn(D.rh[lo], D.rh[hi]));
          const double ex = D.x[hi] - D.x[lo], ey = D.y[hi] - D.y[lo], ez = D.z[hi] - D.z[lo];
          const float w = (float)g0_weight(c, R0, sqrt(fma(ez, ez, fma(ey, ey, ex * ex))));
          sj *= w;
          si *= w;
        }
      }
    }
    if (!valid) { sj = 0.f; si = 0.f; }
    kahan(sxi, cxi, sj * dx); kahan(syi, cyi, sj * dy); kahan(szi, czi, sj * dz);
    kahan(sxj, cxj, -si * dx); kahan(syj, cyj, -si * dy); kahan(szj, czj, -si * dz);
    if (!diag || s + 1 < nsteps) rotate();
  }
  float2 *out = reinterpret_cast<float2 *>(D.part) + (size_t)t * 2 * 3 * 32 + lane;
  if (diag) {
    const int src = (lane + 16) & 31;
    const float hx = __shfl_sync(FULL, sxj, src), hy = __shfl_sync(FULL, syj, src), hz = __shfl_sync(FULL, szj, src);
    const float kx = __shfl_sync(FULL, cxj, src), ky = __shfl_sync(FULL, cyj, src), kz = __shfl_sync(FULL, czj, src);
    kahan(sxi, cxi, hx); kahan(sxi, cxi, -kx);
    kahan(syi, cyi, hy); kahan(syi, cyi, -ky);
    kahan(szi, czi, hz); kahan(szi, czi, -kz);
    out[0] = make_float2(sxi, cxi); out[32] = make_float2(syi, cyi); out[64] = make_float2(szi, czi);
  } else {
    out[0] = make_float2(sxi, cxi); out[32] = make_float2(syi, cyi); out[64] = make_float2(szi, czi);
    out[96] = make_float2(sxj, cxj); out[128] = make_float2(syj, cyj); out[160] = make_float2(szj, czj);
  }
}

template <int MODE>
__global__ void __launch_bounds__(128) k_trap_mixed(Dev D) {
  const int lane = threadIdx.x & 31;
  const int ntiles = D.ntiles_total;
  const int S = D.seg_len;
  int *counter = &D.work[MODE - 1];
  for (;;) {
    int seg = 0;
    if (lane == 0) seg = atomicAdd(counter, 1);
    seg = __shfl_sync(FULL, seg, 0);
    const int t0 = seg * S;
    if (t0 >= ntiles) break;
    const int t1 = min(t0 + S, ntiles);
    for (int t = t0; t < t1; ++t) {
      const int4 tl = D.tiles[t];
      const TileCtx c = load_ctx(&D.disks[tl.x]);
      tile_mixed<MODE>(D, c, t, tl, lane);
    }
  }
}

template <int MODE>
__global__ void __launch_bounds__(128) k_trap_fp64(Dev D) {
  const int lane = threadIdx.x & 31;
  const int ntiles = D.ntiles_total;
  const int S = D.seg_len;
  int *counter = &D.work[MODE - 1];
  for (;;) {
    int seg = 0;
    if (lane == 0) seg = atomicAdd(counter, 1);
    seg = __shfl_sync(FULL, seg, 0);
    const int t0 = seg * S;
    if (t0 >= ntiles) break;
    const int t1 = min(t0 + S, ntiles);
    for (int t = t0; t < t1; ++t) {
      const int4 tl = D.tiles[t];
      const DiskDesc *dp = &D.disks[tl.x];
      const TileCtx c = load_ctx(dp);
      tile_fp64<MODE>(D, c, dp, t, tl, lane);
    }
  }
}

int trap_blocks_per_sm(int precision) {
  int nb = 0;
  if (precision == SYMBA_PRECISION_MIXED) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_trap_mixed<1>, 128, 0);
    if (nb > 8) nb = 8;
  } else {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_trap_fp64<1>, 128, 0);
    if (nb > 4) nb = 4;
  }
  return nb > 0 ? nb : 1;
}

void launch_trap(const Dev &D, const LaunchCfg &L, int mode, int precision, cudaStream_t s) {
  if (D.ntiles_total <= 0) return;
  if (precision == SYMBA_PRECISION_MIXED) {
    if (mode == 1) k_trap_mixed<1><<<L.trap_blocks, 128, 0, s>>>(D);
    else k_trap_mixed<2><<<L.trap_blocks, 128, 0, s>>>(D);
  } else {
    if (mode == 1) k_trap_fp64<1><<<L.trap_blocks, 128, 0, s>>>(D);
    else k_trap_fp64<2><<<L.trap_blocks, 128, 0, s>>>(D);
  }
}

// ---------------------------------------------------------------------------------------------
// The field rectangle (Sec. 2: field particles interact only with massive bodies).  The
// trapezoid's tiles cover the column blocks that hold massive bodies; every block of field
// particles beyond them is one row of the rectangle N_m x N_field, taken by one warp: lane l
// owns field particle b*32 + l, the system's massive bodies stream through a per-warp
// shared-memory chunk of 32 (one coalesced load, then broadcast reads), and only the field
// particle's side is accumulated -- a massless body exerts no force, so the massive side and the
// per-tile partials of the trapezoid are not needed.  The sum over i runs in ascending order,
// so the result does not depend on the launch or on other systems, and the kick
// v += (tau/2) a is applied at the end (the reduction skips these blocks).  Kick 1 runs the same
// fused encounter check as the tiles (FP32 prefilter, exact FP64 predicate, pair emission,
// g_0 weight); kick 2 weights the flagged pairs through the groups.
// ---------------------------------------------------------------------------------------------
struct FieldSrc {
  double x, y, z, gm;
  float xf, yf, zf, xl, yl, zl, gmf;           // FP32 copies; low parts and G m (mixed)
  float vxf, vyf, vzf, lam, sig;               // kick 1 prefilter
  int id, ok, gid;
};

// stage massive bodies [c0, c0 + 32) of the system into the warp's chunk
template <int MODE, bool MIXED>
__device__ __forceinline__ void stage_sources(const Dev &D, const TileCtx &c, int c0, int lane, FieldSrc *src) {
  const int li = c0 + lane;
  FieldSrc s;
  const int p = c.off + li;
  s.id = p;
  s.ok = (li < c.nm && D.alive[p]) ? 1 : 0;
  const int q = s.ok ? p : c.off;               // a valid address for the loads below
  s.x = D.x[q]; s.y = D.y[q]; s.z = D.z[q]; s.gm = D.gm[q];
  s.xf = D.xf[q]; s.yf = D.yf[q]; s.zf = D.zf[q];
  s.xl = 0.f; s.yl = 0.f; s.zl = 0.f; s.gmf = 0.f;
  if (MIXED) {
    s.xl = D.xl[q]; s.yl = D.yl[q]; s.zl = D.zl[q]; s.gmf = D.gmf[q];
  }
  s.vxf = 0.f; s.vyf = 0.f; s.vzf = 0.f; s.lam = 0.f; s.sig = 0.f;
  if (MODE == 1) {
    s.vxf = D.vxf[q]; s.vyf = D.vyf[q]; s.vzf = D.vzf[q]; s.lam = D.lamf[q]; s.sig = D.sigf[q];
  }
  s.gid = MODE == 2 ? D.gid[q] : -1;
  src[lane] = s;
}

// the FP64 predicate of pair (i massive, p field) and, when flagged, its pair-list entry and
// level-0 weight (1 when not flagged)
__device__ __forceinline__ double field_check(const Dev &D, const TileCtx &c, int sys, int i, int p) {
  const double ex = __dsub_rn(D.x[p], D.x[i]), ey = __dsub_rn(D.y[p], D.y[i]), ez = __dsub_rn(D.z[p], D.z[i]);
  const double evx = __dsub_rn(D.vx[p], D.vx[i]), evy = __dsub_rn(D.vy[p], D.vy[i]),
               evz = __dsub_rn(D.vz[p], D.vz[i]);
  const double R0 = __dmul_rn(c.lam, __dadd_rn(D.rh[i], D.rh[p]));
  if (!encounter_exact(ex, ey, ez, evx, evy, evz, R0, c.dt)) return 1.0;
  const int k = atomicAdd(&D.stat[sys].npairs, 1);
  if (k < c.pair_cap) {
    D.raw_i[c.pair_base + k] = i;
    D.raw_j[c.pair_base + k] = p;
  }
  const double er2 = __dadd_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)), __dmul_rn(ez, ez));
  return g0_weight(c, R0, __dsqrt_rn(er2));
}

template <int MODE>
__global__ void __launch_bounds__(128) k_field_fp64(Dev D) {
  __shared__ FieldSrc chunk[4][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int e = blockIdx.x * 4 + w;
  if (e >= D.nfblk) return;
  const int2 fb = D.fblk[e];                     // {system, global block}
  const TileCtx c = load_ctx(&D.disks[fb.x]);
  FieldSrc *src = chunk[w];
  const int p = fb.y * 32 + lane;
  const int lp = p - c.off;
  const bool live = lp < c.n && D.alive[p];
  const double xp = D.x[p], yp = D.y[p], zp = D.z[p];
  const float xfp = D.xf[p], yfp = D.yf[p], zfp = D.zf[p];
  float vxfp = 0.f, vyfp = 0.f, vzfp = 0.f, lamp = 0.f, sigp = 0.f;
  int gidp = -1;
  if (MODE == 1) {
    vxfp = D.vxf[p]; vyfp = D.vyf[p]; vzfp = D.vzf[p]; lamp = D.lamf[p]; sigp = D.sigf[p];
  } else {
    gidp = D.gid[p];
  }
  const float tauf = __double2float_ru(c.dt);
  double ax = 0.0, ay = 0.0, az = 0.0;
  for (int c0 = 0; c0 < c.nm; c0 += 32) {
    __syncwarp();
    stage_sources<MODE, false>(D, c, c0, lane, src);
    __syncwarp();
    const int cnt = min(32, c.nm - c0);
#pragma unroll 1
    for (int s = 0; s < cnt; ++s) {
      const FieldSrc &q = src[s];
      const bool valid = live && q.ok;
      const double dx = q.x - xp, dy = q.y - yp, dz = q.z - zp;
      const double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
      double sp = q.gm * rinv3(r2);
      if (MODE == 1) {
        const float dxf = q.xf - xfp, dyf = q.yf - yfp, dzf = q.zf - zfp;
        const float r2f = fmaf(dzf, dzf, fmaf(dyf, dyf, dxf * dxf));
        const float dvxf = q.vxf - vxfp, dvyf = q.vyf - vyfp, dvzf = q.vzf - vzfp;
        const float vmag = sqrtf(fmaf(dvzf, dvzf, fmaf(dvyf, dvyf, dvxf * dvxf)));
        const float Bf = fmaf(tauf, vmag, q.lam + lamp) * 1.0000039f + 1.9073486e-6f * (q.sig + sigp);
        const bool cand = valid && !(r2f > Bf * Bf);
        if (__any_sync(FULL, cand)) {
          if (cand) sp *= field_check(D, c, fb.x, q.id, p);
        }
      } else if (gidp >= 0 && gidp == q.gid && valid) {
        if (group_has_pair(D, gidp, q.id, p)) {
          const double R0 = __dmul_rn(c.lam, __dadd_rn(D.rh[q.id], D.rh[p]));
          sp *= g0_weight(c, R0, sqrt(r2));
        }
      }
      sp = keep_or_zero(sp, valid);
      ax = fma(sp, dx, ax); ay = fma(sp, dy, ay); az = fma(sp, dz, az);
    }
  }
  if (live) {
    const double h = 0.5 * c.dt;
    D.vx[p] = __dadd_rn(D.vx[p], __dmul_rn(h, ax));
    D.vy[p] = __dadd_rn(D.vy[p], __dmul_rn(h, ay));
    D.vz[p] = __dadd_rn(D.vz[p], __dmul_rn(h, az));
  }
}

// Mixed precision: the same rectangle with the FP32 pair arithmetic of tile_mixed (two-float
// displacement, FP32 rsqrt and one Newton step, Kahan-compensated FP32 sums carried into FP64
// once); the encounter check is the FP64 one.
template <int MODE>
__global__ void __launch_bounds__(128) k_field_mixed(Dev D) {
  __shared__ FieldSrc chunk[4][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int e = blockIdx.x * 4 + w;
  if (e >= D.nfblk) return;
  const int2 fb = D.fblk[e];
  const TileCtx c = load_ctx(&D.disks[fb.x]);
  FieldSrc *src = chunk[w];
  const int p = fb.y * 32 + lane;
  const int lp = p - c.off;
  const bool live = lp < c.n && D.alive[p];
  const float xhp = D.xf[p], yhp = D.yf[p], zhp = D.zf[p];
  const float xlp = D.xl[p], ylp = D.yl[p], zlp = D.zl[p];
  float vxfp = 0.f, vyfp = 0.f, vzfp = 0.f, lamp = 0.f, sigp = 0.f;
  int gidp = -1;
  if (MODE == 1) {
    vxfp = D.vxf[p]; vyfp = D.vyf[p]; vzfp = D.vzf[p]; lamp = D.lamf[p]; sigp = D.sigf[p];
  } else {
    gidp = D.gid[p];
  }
  const float tauf = __double2float_ru(c.dt);
  float sx = 0.f, sy = 0.f, sz = 0.f, cx = 0.f, cy = 0.f, cz = 0.f;
  for (int c0 = 0; c0 < c.nm; c0 += 32) {
    __syncwarp();
    stage_sources<MODE, true>(D, c, c0, lane, src);
    __syncwarp();
    const int cnt = min(32, c.nm - c0);
#pragma unroll 1
    for (int s = 0; s < cnt; ++s) {
      const FieldSrc &q = src[s];
      const bool valid = live && q.ok;
      const float dx = (q.xf - xhp) + (q.xl - xlp);
      const float dy = (q.yf - yhp) + (q.yl - ylp);
      const float dz = (q.zf - zhp) + (q.zl - zlp);
      const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
      float ri;
      asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(ri) : "f"(r2));
      ri = ri * fmaf(-0.5f * r2, ri * ri, 1.5f);
      float sp = q.gmf * (ri * ri * ri);
      if (MODE == 1) {
        const float dvxf = q.vxf - vxfp, dvyf = q.vyf - vyfp, dvzf = q.vzf - vzfp;
        const float vmag = sqrtf(fmaf(dvzf, dvzf, fmaf(dvyf, dvyf, dvxf * dvxf)));
        const float Bf = fmaf(tauf, vmag, q.lam + lamp) * 1.0000039f + 1.9073486e-6f * (q.sig + sigp);
        const bool cand = valid && !(r2 > Bf * Bf * 1.0000153f);
        if (__any_sync(FULL, cand)) {
          if (cand) sp *= (float)field_check(D, c, fb.x, q.id, p);
        }
      } else if (gidp >= 0 && gidp == q.gid && valid) {
        if (group_has_pair(D, gidp, q.id, p)) {
          const double R0 = __dmul_rn(c.lam, __dadd_rn(D.rh[q.id], D.rh[p]));
          const double ex = D.x[p] - D.x[q.id], ey = D.y[p] - D.y[q.id], ez = D.z[p] - D.z[q.id];
          sp *= (float)g0_weight(c, R0, sqrt(fma(ez, ez, fma(ey, ey, ex * ex))));
        }
      }
      if (!valid) sp = 0.f;
      kahan(sx, cx, sp * dx); kahan(sy, cy, sp * dy); kahan(sz, cz, sp * dz);
    }
  }
  if (live) {
    const double h = 0.5 * c.dt;
    D.vx[p] = fma(h, (double)sx - (double)cx, D.vx[p]);
    D.vy[p] = fma(h, (double)sy - (double)cy, D.vy[p]);
    D.vz[p] = fma(h, (double)sz - (double)cz, D.vz[p]);
  }
}

void launch_field(const Dev &D, int mode, int precision, cudaStream_t s) {
  if (D.nfblk <= 0) return;
  const int blocks = (D.nfblk + 3) / 4;
  if (precision == SYMBA_PRECISION_MIXED) {
    if (mode == 1) k_field_mixed<1><<<blocks, 128, 0, s>>>(D);
    else k_field_mixed<2><<<blocks, 128, 0, s>>>(D);
  } else {
    if (mode == 1) k_field_fp64<1><<<blocks, 128, 0, s>>>(D);
    else k_field_fp64<2><<<blocks, 128, 0, s>>>(D);
  }
}
