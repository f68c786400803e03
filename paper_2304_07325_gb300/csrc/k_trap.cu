// The right-angled-trapezoid pair kick (Sec. 2): every pair i < N_m, j > i once, both
// reactions accumulated, no atomics.
//
// Work decomposition.  Indices are cut into 32-blocks; tile (I, J), I <= J, over the column
// blocks that hold massive bodies, holds the pairs of block I (rows) with block J (columns): the
// trapezoid becomes a rectangle of off-diagonal tiles plus the diagonal tiles of the triangle.
// Tiles are grouped into macro-tiles of 4 row blocks (a 128-body quad q) by SYM_MACRO_COLS column
// blocks (column group p, p >= 4q / SYM_MACRO_COLS), all macro-tiles of all systems in one flat
// list that persistent CTAs of four warps consume from a counter (the fold of the triangle into a
// rectangle, done by a work queue instead of index arithmetic).
//
// One CTA per macro-tile, one warp per row block: warp w keeps row particle (4q + w)*32 + l in
// lane l and sweeps the macro's column blocks in turn; in each tile lane l meets column
// (l + s) mod 32 at step s (32 steps; 16 on a diagonal tile, where each unordered pair is met
// once).  In the FP64 path the tile's column bodies are staged in the warp's shared memory and
// only their accumulators rotate through the lanes by warp shuffle; the mixed path rotates the
// bodies with them.  After the sweep every column accumulator is back in its home lane.  The row accumulators run on across the
// macro-tile's tiles and are written once per macro-tile; the four warps' column accumulators of
// each column block are added in shared memory in warp order and written once.  Both kinds of partials are
// summed later in a fixed order: the result does not depend on scheduling, on how many
// macro-tiles a CTA takes per grab, or on which other systems share the launch.
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


// partial slots of macro-tile m: rows [w][component][lane], then columns [k][component][lane]
__device__ __forceinline__ size_t part_row(int m, int w) { return (size_t)m * SYM_MACRO_PART + w * 96; }
__device__ __forceinline__ size_t part_col(int m, int k) { return (size_t)m * SYM_MACRO_PART + 384 + k * 96; }
#define MC SYM_MACRO_COLS

// the row side of one warp: row particle I*32 + lane, its data and its accumulators
struct RowF64 {
  int pi;
  bool live, row;          // a live body; live and massive (a row of the trapezoid)
  double x, y, z, ngm;     // position and -G m of the row body
  float xf, yf, zf, vxf, vyf, vzf, lam, sig;   // kick 1: FP32 prefilter copies
  int gid;                 // kick 2: encounter group
  double ax, ay, az;       // carried across the macro-tile's column blocks
};

template <int MODE>
__device__ __forceinline__ void row_load_fp64(const Dev &D, const TileCtx &c, int I, int lane, RowF64 &r) {
  r.pi = I * 32 + lane;
  const int li = r.pi - c.off;
  r.live = li < c.n && D.alive[r.pi];
  r.row = r.live && li < c.nm;
  r.x = D.x[r.pi]; r.y = D.y[r.pi]; r.z = D.z[r.pi];
  r.ngm = __longlong_as_double(__double_as_longlong(D.gm[r.pi]) ^ (long long)0x8000000000000000ull);
  r.xf = r.yf = r.zf = r.vxf = r.vyf = r.vzf = r.lam = r.sig = 0.f;
  r.gid = -1;
  if (MODE == 1) {
    r.xf = D.xf[r.pi]; r.yf = D.yf[r.pi]; r.zf = D.zf[r.pi];
    r.vxf = D.vxf[r.pi]; r.vyf = D.vyf[r.pi]; r.vzf = D.vzf[r.pi];
    r.lam = D.lamf[r.pi]; r.sig = D.sigf[r.pi];
  } else {
    r.gid = D.gid[r.pi];
  }
  r.ax = r.ay = r.az = 0.0;
}

// One warp's copy of a tile's 32 column bodies in shared memory.
struct JStage {
  double2 xy[32], zg[32];   // x, y | z, G m
  float4 fa[32], fb[32];    // kick 1: the FP32 copies xf, yf, zf, vxf | vyf, vzf, lambda, sigma
  int gid[32];              // kick 2: encounter group
};

// One 32 x 32 tile (rows of block I, columns of block J >= I): both reactions of every pair;
// the row side goes into r.ax.., the column side comes back in cx, cy, cz (zero on a diagonal
// tile, whose column side is folded into its rows).  The column bodies are staged in js once;
// at step s lane l takes column (l + s + o) mod 32 (o = 1 on a diagonal tile), whose column-side
// sums travel with it from lane to lane.
template <int MODE>
__device__ __forceinline__ void tile_sweep_fp64(const Dev &D, const TileCtx &c, int sys, RowF64 &r,
                                                int I, int J, int lane, JStage *js, double &cx,
                                                double &cy, double &cz) {
  const bool diag = I == J;
  {
    const int j0 = J * 32 + lane;
    __syncwarp();                         // the last tile's reads of js are done
    js->xy[lane] = make_double2(D.x[j0], D.y[j0]);
    js->zg[lane] = make_double2(D.z[j0], D.gm[j0]);
    if (MODE == 1) {
      js->fa[lane] = make_float4(D.xf[j0], D.yf[j0], D.zf[j0], D.vxf[j0]);
      js->fb[lane] = make_float4(D.vyf[j0], D.vzf[j0], D.lamf[j0], D.sigf[j0]);
    } else {
      js->gid[lane] = D.gid[j0];
    }
  }
  const int lj0 = J * 32 + lane - c.off;
  const bool live_j0 = lj0 < c.n && D.alive[J * 32 + lane];
  const unsigned mlive = __ballot_sync(FULL, live_j0), mmass = __ballot_sync(FULL, live_j0 && lj0 < c.nm);
  __syncwarp();
  double axj = 0.0, ayj = 0.0, azj = 0.0;
  const float tauf = __double2float_ru(c.dt);

  auto rotate = [&]() {
    const int src = (lane + 1) & 31;
    axj = __shfl_sync(FULL, axj, src); ayj = __shfl_sync(FULL, ayj, src);
    azj = __shfl_sync(FULL, azj, src);
  };

  const int nsteps = diag ? 16 : 32, o = diag ? 1 : 0;
#pragma unroll 1
  for (int s = 0; s < nsteps; ++s) {
    const int cj = (lane + s + o) & 31;
    const int jid = J * 32 + cj;
    const int jflags = (int)((mlive >> cj) & 1u) | (int)(((mmass >> cj) & 1u) << 1);
    const double2 q0 = js->xy[cj], q1 = js->zg[cj];
    const double xj = q0.x, yj = q0.y, zj = q1.x, gmj = q1.y;
    float xfj = 0.f, yfj = 0.f, zfj = 0.f, vxfj = 0.f, vyfj = 0.f, vzfj = 0.f, lamj = 0.f, sigj = 0.f;
    int gidj = -1;
    if (MODE == 1) {
      const float4 fa = js->fa[cj], fb = js->fb[cj];
      xfj = fa.x; yfj = fa.y; zfj = fa.z; vxfj = fa.w;
      vyfj = fb.x; vzfj = fb.y; lamj = fb.z; sigj = fb.w;
    } else {
      gidj = js->gid[cj];
    }
    bool valid;
    if (!diag) {
      valid = r.row && (jflags & 1);
    } else {
      valid = (jid > r.pi) ? (r.row && (jflags & 1)) : (r.live && (jflags & 2));
      if (s == 15 && lane >= 16) valid = false;  // pair {l, l+16} belongs to lane l < 16
    }
    const double dx = xj - r.x, dy = yj - r.y, dz = zj - r.z;
    const double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
    const double r3 = rinv3(r2);
    double sj = gmj * r3;
    double si = r.ngm * r3;             // the column side's -G m_i / r^3
    if (MODE == 1) {
      const float dxf = xfj - r.xf, dyf = yfj - r.yf, dzf = zfj - r.zf;
      const float r2f = fmaf(dzf, dzf, fmaf(dyf, dyf, dxf * dxf));
      const float dvxf = vxfj - r.vxf, dvyf = vyfj - r.vyf, dvzf = vzfj - r.vzf;
      const float vmag = sqrtf(fmaf(dvzf, dvzf, fmaf(dvyf, dvyf, dvxf * dvxf)));
      const float Bf = fmaf(tauf, vmag, r.lam + lamj) * 1.0000039f + 1.9073486e-6f * (r.sig + sigj);
      const bool cand = valid && !(r2f > Bf * Bf);
      if (__any_sync(FULL, cand)) {
        if (cand) {
          const int lo = min(r.pi, jid), hi = max(r.pi, jid);
          const double ex = __dsub_rn(D.x[hi], D.x[lo]), ey = __dsub_rn(D.y[hi], D.y[lo]),
                       ez = __dsub_rn(D.z[hi], D.z[lo]);
          const double evx = __dsub_rn(D.vx[hi], D.vx[lo]), evy = __dsub_rn(D.vy[hi], D.vy[lo]),
                       evz = __dsub_rn(D.vz[hi], D.vz[lo]);
          const double R0 = __dmul_rn(c.lam, __dadd_rn(D.rh[lo], D.rh[hi]));
          if (encounter_exact(ex, ey, ez, evx, evy, evz, R0, c.dt)) {
            const int k = atomicAdd(&D.stat[sys].npairs, 1);
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
      if (r.gid >= 0 && r.gid == gidj && valid) {
        const int lo = min(r.pi, jid), hi = max(r.pi, jid);
        if (group_has_pair(D, r.gid, lo, hi)) {
          const double R0 = __dmul_rn(c.lam, __dadd_rn(D.rh[lo], D.rh[hi]));
          const double w = g0_weight(c, R0, sqrt(r2));
          sj *= w;
          si *= w;
        }
      }
    }
    sj = keep_or_zero(sj, valid);
    si = keep_or_zero(si, valid);
    r.ax = fma(sj, dx, r.ax); r.ay = fma(sj, dy, r.ay); r.az = fma(sj, dz, r.az);
    axj = fma(si, dx, axj); ayj = fma(si, dy, ayj); azj = fma(si, dz, azj);
    if (!diag || s + 1 < nsteps) rotate();
  }
  if (diag) {
    const int src = (lane + 16) & 31;
    r.ax += __shfl_sync(FULL, axj, src);
    r.ay += __shfl_sync(FULL, ayj, src);
    r.az += __shfl_sync(FULL, azj, src);
    cx = 0.0; cy = 0.0; cz = 0.0;
  } else {
    cx = axj; cy = ayj; cz = azj;
  }
}

// Mixed precision (FP32 pair path): the relative displacement is formed from the two-float split
// x = xf + xl of each FP64 position, (xf_j - xf_i) + (xl_j - xl_i) -- RN32 of the FP64 difference
// or a neighbouring float for every pair the level-0 weight does not zero; r^-3 from the FP32
// rsqrt plus one Newton step; both sides accumulated in FP32 with Kahan compensation and written
// as (sum, compensation) pairs that the reduction carries into FP64.  The encounter check is the
// same FP64 decision as in the FP64 path.
__device__ __forceinline__ void kahan(float &s, float &c, float term) {
  const float y = term - c;
  const float t = s + y;
  c = (t - s) - y;
  s = t;
}

struct RowMixed {
  int pi;
  bool live, row;
  float xh, yh, zh, xl, yl, zl, gm;
  float vxf, vyf, vzf, lam, sig;   // kick 1 prefilter
  int gid;                         // kick 2
  float sx, sy, sz, cx, cy, cz;    // Kahan sums of the row side, carried across the macro-tile
};

template <int MODE>
__device__ __forceinline__ void row_load_mixed(const Dev &D, const TileCtx &c, int I, int lane, RowMixed &r) {
  r.pi = I * 32 + lane;
  const int li = r.pi - c.off;
  r.live = li < c.n && D.alive[r.pi];
  r.row = r.live && li < c.nm;
  r.xh = D.xf[r.pi]; r.yh = D.yf[r.pi]; r.zh = D.zf[r.pi];
  r.xl = D.xl[r.pi]; r.yl = D.yl[r.pi]; r.zl = D.zl[r.pi];
  r.gm = D.gmf[r.pi];
  r.vxf = r.vyf = r.vzf = r.lam = r.sig = 0.f;
  r.gid = -1;
  if (MODE == 1) {
    r.vxf = D.vxf[r.pi]; r.vyf = D.vyf[r.pi]; r.vzf = D.vzf[r.pi]; r.lam = D.lamf[r.pi]; r.sig = D.sigf[r.pi];
  } else {
    r.gid = D.gid[r.pi];
  }
  r.sx = r.sy = r.sz = r.cx = r.cy = r.cz = 0.f;
}

// one tile; the column side comes back as Kahan pairs (s, c) per component, zero on a diagonal
template <int MODE>
__device__ __forceinline__ void tile_sweep_mixed(const Dev &D, const TileCtx &c, int sys, RowMixed &r,
                                                 int I, int J, int lane, float2 &ox, float2 &oy, float2 &oz) {
  const bool diag = I == J;
  int jid = J * 32 + lane;
  const int lj0 = jid - c.off;
  const bool live_j0 = lj0 < c.n && D.alive[jid];
  int jflags = (live_j0 ? 1 : 0) | ((live_j0 && lj0 < c.nm) ? 2 : 0);
  float xhj = D.xf[jid], yhj = D.yf[jid], zhj = D.zf[jid];
  float xlj = D.xl[jid], ylj = D.yl[jid], zlj = D.zl[jid];
  float gmj = D.gmf[jid];
  float sxj = 0.f, syj = 0.f, szj = 0.f, cxj = 0.f, cyj = 0.f, czj = 0.f;
  float vxfj = 0.f, vyfj = 0.f, vzfj = 0.f, lamj = 0.f, sigj = 0.f;
  int gidj = -1;
  if (MODE == 1) {
    vxfj = D.vxf[jid]; vyfj = D.vyf[jid]; vzfj = D.vzf[jid]; lamj = D.lamf[jid]; sigj = D.sigf[jid];
  } else {
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
      valid = r.row && (jflags & 1);
    } else {
      valid = (jid > r.pi) ? (r.row && (jflags & 1)) : (r.live && (jflags & 2));
      if (s == 15 && lane >= 16) valid = false;
    }
    const float dx = (xhj - r.xh) + (xlj - r.xl);
    const float dy = (yhj - r.yh) + (ylj - r.yl);
    const float dz = (zhj - r.zh) + (zlj - r.zl);
    const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
    float ri;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(ri) : "f"(r2));
    ri = ri * fmaf(-0.5f * r2, ri * ri, 1.5f);
    const float s3 = ri * ri * ri;
    float sj = gmj * s3, si = r.gm * s3;
    if (MODE == 1) {
      const float dvxf = vxfj - r.vxf, dvyf = vyfj - r.vyf, dvzf = vzfj - r.vzf;
      const float vmag = sqrtf(fmaf(dvzf, dvzf, fmaf(dvyf, dvyf, dvxf * dvxf)));
      const float Bf = fmaf(tauf, vmag, r.lam + lamj) * 1.0000039f + 1.9073486e-6f * (r.sig + sigj);
      const bool cand = valid && !(r2 > Bf * Bf * 1.0000153f);
      if (__any_sync(FULL, cand)) {
        if (cand) {
          const int lo = min(r.pi, jid), hi = max(r.pi, jid);
          const double ex = __dsub_rn(D.x[hi], D.x[lo]), ey = __dsub_rn(D.y[hi], D.y[lo]),
                       ez = __dsub_rn(D.z[hi], D.z[lo]);
          const double evx = __dsub_rn(D.vx[hi], D.vx[lo]), evy = __dsub_rn(D.vy[hi], D.vy[lo]),
                       evz = __dsub_rn(D.vz[hi], D.vz[lo]);
          const double R0 = __dmul_rn(c.lam, __dadd_rn(D.rh[lo], D.rh[hi]));
          if (encounter_exact(ex, ey, ez, evx, evy, evz, R0, c.dt)) {
            const int k = atomicAdd(&D.stat[sys].npairs, 1);
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
      if (r.gid >= 0 && r.gid == gidj && valid) {
        const int lo = min(r.pi, jid), hi = max(r.pi, jid);
        if (group_has_pair(D, r.gid, lo, hi)) {
          const double R0 = __dmul_rn(c.lam, __dadd_rn(D.rh[lo], D.rh[hi]));
          const double ex = D.x[hi] - D.x[lo], ey = D.y[hi] - D.y[lo], ez = D.z[hi] - D.z[lo];
          const float w = (float)g0_weight(c, R0, sqrt(fma(ez, ez, fma(ey, ey, ex * ex))));
          sj *= w;
          si *= w;
        }
      }
    }
    if (!valid) { sj = 0.f; si = 0.f; }
    kahan(r.sx, r.cx, sj * dx); kahan(r.sy, r.cy, sj * dy); kahan(r.sz, r.cz, sj * dz);
    kahan(sxj, cxj, -si * dx); kahan(syj, cyj, -si * dy); kahan(szj, czj, -si * dz);
    if (!diag || s + 1 < nsteps) rotate();
  }
  if (diag) {
    const int src = (lane + 16) & 31;
    const float hx = __shfl_sync(FULL, sxj, src), hy = __shfl_sync(FULL, syj, src), hz = __shfl_sync(FULL, szj, src);
    const float kx = __shfl_sync(FULL, cxj, src), ky = __shfl_sync(FULL, cyj, src), kz = __shfl_sync(FULL, czj, src);
    kahan(r.sx, r.cx, hx); kahan(r.sx, r.cx, -kx);
    kahan(r.sy, r.cy, hy); kahan(r.sy, r.cy, -ky);
    kahan(r.sz, r.cz, hz); kahan(r.sz, r.cz, -kz);
    ox = make_float2(0.f, 0.f); oy = ox; oz = ox;
  } else {
    ox = make_float2(sxj, cxj); oy = make_float2(syj, cyj); oz = make_float2(szj, czj);
  }
}

// One CTA (four warps) per macro-tile.  The macro-tile list entry is {system, first row block,
// first column block, end of the system's massive blocks}; warp w takes row block I0 + w and
// sweeps column blocks J0..J0+SYM_MACRO_COLS-1, skipping those below its row (the triangle) or
// past the massive blocks.  Rows are written once per macro-tile, columns after the four warps' sums for
// each column block are added in warp order through shared memory.
template <int MODE>
__global__ void __launch_bounds__(128) k_trap_fp64(Dev D) {
  __shared__ double colbuf[4][MC][3][32];     // [warp][column block][component][lane]
  __shared__ JStage jstage[4];
  __shared__ int s_item;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int nmac = D.ntiles_total;
  const int S = D.seg_len;
  int *counter = &D.work[MODE - 1];
  if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
  __syncthreads();
  int m0 = s_item * S;
  while (m0 < nmac) {
    const int m1 = min(m0 + S, nmac);
    for (int m = m0; m < m1; ++m) {
      const int4 mt = D.tiles[m];
      const TileCtx c = load_ctx(&D.disks[mt.x]);
      const int I = mt.y + w;
      const bool has_row = I < mt.w;
      RowF64 r;
      if (has_row) row_load_fp64<MODE>(D, c, I, lane, r);
#pragma unroll 1
      for (int k = 0; k < MC; ++k) {
        const int J = mt.z + k;
        double cx = 0.0, cy = 0.0, cz = 0.0;
        if (has_row && J < mt.w && J >= I)
          tile_sweep_fp64<MODE>(D, c, mt.x, r, I, J, lane, &jstage[w], cx, cy, cz);
        colbuf[w][k][0][lane] = cx; colbuf[w][k][1][lane] = cy; colbuf[w][k][2][lane] = cz;
      }
      double *rowp = D.part + part_row(m, w) + lane;
      rowp[0] = has_row ? r.ax : 0.0; rowp[32] = has_row ? r.ay : 0.0; rowp[64] = has_row ? r.az : 0.0;
      __syncthreads();
      if (w < MC) {                                             // warp w adds column block w
        double *colp = D.part + part_col(m, w) + lane;
#pragma unroll
        for (int q = 0; q < 3; ++q)
          colp[32 * q] = ((colbuf[0][w][q][lane] + colbuf[1][w][q][lane]) + colbuf[2][w][q][lane]) + colbuf[3][w][q][lane];
      }
      // the next item is taken while the columns are added (everyone has read s_item)
      if (m + 1 == m1 && threadIdx.x == 0) s_item = atomicAdd(counter, 1);
      __syncthreads();                        // colbuf is free, s_item is current
    }
    m0 = s_item * S;
  }
}

template <int MODE>
__global__ void __launch_bounds__(128) k_trap_mixed(Dev D) {
  __shared__ float2 colbuf[4][MC][3][32];
  __shared__ int s_item;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int nmac = D.ntiles_total;
  const int S = D.seg_len;
  int *counter = &D.work[MODE - 1];
  float2 *part = reinterpret_cast<float2 *>(D.part);
  if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
  __syncthreads();
  int m0 = s_item * S;
  while (m0 < nmac) {
    const int m1 = min(m0 + S, nmac);
    for (int m = m0; m < m1; ++m) {
      const int4 mt = D.tiles[m];
      const TileCtx c = load_ctx(&D.disks[mt.x]);
      const int I = mt.y + w;
      const bool has_row = I < mt.w;
      RowMixed r;
      if (has_row) row_load_mixed<MODE>(D, c, I, lane, r);
#pragma unroll 1
      for (int k = 0; k < MC; ++k) {
        const int J = mt.z + k;
        float2 ox = make_float2(0.f, 0.f), oy = ox, oz = ox;
        if (has_row && J < mt.w && J >= I) tile_sweep_mixed<MODE>(D, c, mt.x, r, I, J, lane, ox, oy, oz);
        colbuf[w][k][0][lane] = ox; colbuf[w][k][1][lane] = oy; colbuf[w][k][2][lane] = oz;
      }
      float2 *rowp = part + part_row(m, w) + lane;
      const float2 z = make_float2(0.f, 0.f);
      rowp[0] = has_row ? make_float2(r.sx, r.cx) : z;
      rowp[32] = has_row ? make_float2(r.sy, r.cy) : z;
      rowp[64] = has_row ? make_float2(r.sz, r.cz) : z;
      __syncthreads();
      if (w < MC) {
        float2 *colp = part + part_col(m, w) + lane;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          float s = 0.f, cc = 0.f;
#pragma unroll
          for (int v = 0; v < 4; ++v) {
            const float2 t = colbuf[v][w][q][lane];
            kahan(s, cc, t.x);
            kahan(s, cc, -t.y);
          }
          colp[32 * q] = make_float2(s, cc);
        }
      }
      if (m + 1 == m1 && threadIdx.x == 0) s_item = atomicAdd(counter, 1);
      __syncthreads();
    }
    m0 = s_item * S;
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
