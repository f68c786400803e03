// O(N) kernels of the step: set-up, sun drift, partial-sum reduction with the kick, Kepler drift,
// exact total momentum, state transfer and the energy diagnostic.
#include "internal.cuh"

// --------------------------------------------------------------------------------------------
// per-system set-up: shell factors c_k = c_{k-1} / (R_k/R_{k+1}), c_0 = 1
// --------------------------------------------------------------------------------------------
__global__ void k_setup_disk(Dev D, int d) {
  if (threadIdx.x != 0) return;
  DiskDesc *dd = &D.disks[d];
  double c = 1.0;
  for (int k = 0; k < SYM_MAX_LEVELS + 2; ++k) {
    dd->ck[k] = c;
    dd->ck2[k] = c * c;
    c = c / dd->shell_ratio;
  }
  for (int k = 0; k < SYM_MAX_LEVELS + 1; ++k) dd->invdc[k] = 1.0 / (dd->ck[k] - dd->ck[k + 1]);
  dd->invdc[SYM_MAX_LEVELS + 1] = 0.0;
  DiskStat *st = &D.stat[d];
  st->npairs = 0;
  st->ngroups = 0;
  st->status = 0;
  st->max_depth = 0;
  st->merges = 0;
  st->substeps = 0;
  st->max_chain = 0;
  st->merges_reported = 0;
  st->removals = 0;
  st->pair_substeps = 0;
}

void launch_setup_disk(const Dev &D, int d, cudaStream_t s) { k_setup_disk<<<1, 32, 0, s>>>(D, d); }

// --------------------------------------------------------------------------------------------
// removal after the closing kick: a live body with r^2 = (x^2 + y^2) + z^2 (each operation
// rounded once) below rmin^2 or above rmax^2 leaves the system the way a body merged away does
// (mass, G m, radius and Hill radius 0, flag 0), before the total momentum of the closing sun
// drift is summed
// --------------------------------------------------------------------------------------------
__global__ void k_discard(Dev D, long long npart) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < npart;
       p += (long long)gridDim.x * blockDim.x) {
    const int d = D.blk_disk[p >> 5];
    if (d < 0) continue;
    const DiskDesc &dd = D.disks[d];
    if (!dd.active || !D.alive[p] || (dd.rmin2 <= 0.0 && dd.rmax2 <= 0.0)) continue;
    const double x = D.x[p], y = D.y[p], z = D.z[p];
    const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y)), __dmul_rn(z, z));
    if ((dd.rmin2 > 0.0 && r2 < dd.rmin2) || (dd.rmax2 > 0.0 && r2 > dd.rmax2)) {
      D.m[p] = 0.0;
      D.gm[p] = 0.0;
      D.rad[p] = 0.0;
      D.rh[p] = 0.0;
      D.alive[p] = 0;
      atomicAdd(&D.stat[d].removals, 1ull);
    }
  }
}

void launch_discard(const Dev &D, long long npart, cudaStream_t s) {
  if (npart > 0) k_discard<<<(int)std::min((npart + 255) / 256, 4096LL), 256, 0, s>>>(D, npart);
}

// --------------------------------------------------------------------------------------------
// initial upload: heliocentric -> barycentric velocities with exact sums
//   v_i = v_i^hel - S / (m0 + Mt),  S = sum m_j v_j^hel,  Mt = sum m_j   (each correctly rounded)
// and Hill radii rH_i = a_i (m_i / 3 m0)^{1/3} from the osculating heliocentric orbit
// (vis-viva 1/a = 2/r - v^2/mu, mu = G (m0 + m_i); r if unbound; correctly rounded cube root).
// --------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_init_sums(Dev D, int d, int n, const double *vh,
                                                   const double *m, double *q_out) {
  __shared__ unsigned long long acc[4][SA_NDIG + 1];
  for (int k = threadIdx.x; k < 4 * (SA_NDIG + 1); k += blockDim.x) (&acc[0][0])[k] = 0ull;
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double mi = m[i];
    sa_add(acc[3], mi);
    for (int c = 0; c < 3; ++c) sa_add(acc[c], __dmul_rn(mi, vh[3 * i + c]));
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const DiskDesc dd = D.disks[d];
    const double Mt = sa_round(acc[3]);
    const double denom = __dadd_rn(dd.m0, Mt);
    for (int c = 0; c < 3; ++c) q_out[c] = __ddiv_rn(sa_round(acc[c]), denom);
  }
}

__global__ void k_init_state(Dev D, int d, int n, const double *xh, const double *vh,
                             const double *m, const double *rad, const double *rh,
                             int compute_rh, const double *q) {
  const DiskDesc dd = D.disks[d];
  const int npad = dd.nb * SYM_TILE;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < npad; i += gridDim.x * blockDim.x) {
    const int p = dd.off + i;
    if (i < n) {
      const double x = xh[3 * i], y = xh[3 * i + 1], z = xh[3 * i + 2];
      const double ux = vh[3 * i], uy = vh[3 * i + 1], uz = vh[3 * i + 2];
      D.x[p] = x; D.y[p] = y; D.z[p] = z;
      D.vx[p] = __dsub_rn(ux, q[0]);
      D.vy[p] = __dsub_rn(uy, q[1]);
      D.vz[p] = __dsub_rn(uz, q[2]);
      const double mi = m[i];
      D.m[p] = mi;
      D.gm[p] = __dmul_rn(dd.G, mi);
      D.rad[p] = rad[i];
      double h;
      if (compute_rh) {
        const double r = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y)), __dmul_rn(z, z)));
        const double v2 = __dadd_rn(__dadd_rn(__dmul_rn(ux, ux), __dmul_rn(uy, uy)), __dmul_rn(uz, uz));
        const double mu = __dmul_rn(dd.G, __dadd_rn(dd.m0, mi));
        const double inv_a = __dsub_rn(__ddiv_rn(2.0, r), __ddiv_rn(v2, mu));
        const double a = inv_a > 0.0 ? __ddiv_rn(1.0, inv_a) : r;
        h = __dmul_rn(a, cbrt_rn(__ddiv_rn(mi, __dmul_rn(3.0, dd.m0))));
      } else {
        h = rh[i];
      }
      D.rh[p] = h;
      D.alive[p] = 1;
    } else {
      // padding: massless, outside the system, far apart from each other
      D.x[p] = 1.0e9 + 1.0e3 * (double)i; D.y[p] = 0.0; D.z[p] = 0.0;
      D.vx[p] = 0.0; D.vy[p] = 0.0; D.vz[p] = 0.0;
      D.m[p] = 0.0; D.gm[p] = 0.0; D.rad[p] = 0.0; D.rh[p] = 0.0;
      D.alive[p] = 0;
    }
    D.gid[p] = -1;
  }
}

void launch_init_state(const Dev &D, int d, int n, const double *xh, const double *vh,
                       const double *m, const double *rad, const double *rh, int compute_rh,
                       cudaStream_t s) {
  // q (3 doubles) lives in the momentum slot of the system until the first momentum pass
  double *q = D.P + 3 * d;
  k_init_sums<<<1, 256, 0, s>>>(D, d, n, vh, m, q);
  k_init_state<<<64, 256, 0, s>>>(D, d, n, xh, vh, m, rad, rh, compute_rh, q);
}

// --------------------------------------------------------------------------------------------
// per-step prologue: reset the per-step counters
// --------------------------------------------------------------------------------------------
__global__ void k_prologue(Dev D, int ndisks) {
  const int t = threadIdx.x;
  if (t < 4) D.work[t] = 0;
  if (t == 0) *D.rec_total = 0;
  for (int d = t; d < ndisks; d += blockDim.x) {
    D.stat[d].npairs = 0;
    D.stat[d].ngroups = 0;
  }
}

void launch_prologue(const Dev &D, int ndisks, cudaStream_t s) { k_prologue<<<1, 256, 0, s>>>(D, ndisks); }

// --------------------------------------------------------------------------------------------
// exact total barycentric momentum P_d = sum m_i v_i of every system: MOM_CTAS CTAs per system
// accumulate their share into shared-memory digits, add the digits to the system's global
// accumulator, and a second pass rounds it and clears it for the next use.
// --------------------------------------------------------------------------------------------
#define MOM_CTAS 24

__global__ void __launch_bounds__(256) k_momentum_acc(Dev D) {
  const int d = blockIdx.y;
  const DiskDesc &dd = D.disks[d];
  if (!dd.active) return;
  __shared__ unsigned long long acc[3][SA_NDIG + 1];
  for (int k = threadIdx.x; k < 3 * (SA_NDIG + 1); k += blockDim.x) (&acc[0][0])[k] = 0ull;
  __syncthreads();
  const int n = dd.n, off = dd.off;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int p = off + i;
    if (!D.alive[p]) continue;
    const double mi = D.m[p];
    if (mi == 0.0) continue;
    sa_add(acc[0], __dmul_rn(mi, D.vx[p]));
    sa_add(acc[1], __dmul_rn(mi, D.vy[p]));
    sa_add(acc[2], __dmul_rn(mi, D.vz[p]));
  }
  __syncthreads();
  unsigned long long *g = D.sacc + (size_t)d * 3 * (SA_NDIG + 1);
  for (int k = threadIdx.x; k < 3 * (SA_NDIG + 1); k += blockDim.x) {
    const unsigned long long v = (&acc[0][0])[k];
    if (v) atomicAdd(&g[k], v);
  }
}

__global__ void k_momentum_round(Dev D) {
  const int d = blockIdx.x;
  if (!D.disks[d].active) return;
  unsigned long long *g = D.sacc + (size_t)d * 3 * (SA_NDIG + 1);
  if (threadIdx.x < 3) D.P[3 * d + threadIdx.x] = sa_round(g + threadIdx.x * (SA_NDIG + 1));
  __syncthreads();
  for (int k = threadIdx.x; k < 3 * (SA_NDIG + 1); k += blockDim.x) g[k] = 0ull;
}

void launch_momentum(const Dev &D, int ndisks, cudaStream_t s) {
  if (ndisks <= 0) return;
  k_momentum_acc<<<dim3(MOM_CTAS, ndisks), 256, 0, s>>>(D);
  k_momentum_round<<<ndisks, 32, 0, s>>>(D);
}

// --------------------------------------------------------------------------------------------
// sun drift h = tau/2: x_i = x_i + h (P / m0), component by component (q = P_c / m0, d = h q).
// The drift that opens a step also writes the FP32 copies the encounter prefilter reads.
// --------------------------------------------------------------------------------------------
__global__ void k_sundrift(Dev D, long long npart, int pre) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < npart;
       p += (long long)gridDim.x * blockDim.x) {
    const int d = D.blk_disk[p >> 5];
    if (d < 0) continue;
    const DiskDesc &dd = D.disks[d];
    if (!dd.active) continue;
    double x = D.x[p], y = D.y[p], z = D.z[p];
    if (D.alive[p]) {
      const double h = 0.5 * dd.dt;
      const double *P = D.P + 3 * d;
      x = __dadd_rn(x, __dmul_rn(h, __ddiv_rn(P[0], dd.m0)));
      y = __dadd_rn(y, __dmul_rn(h, __ddiv_rn(P[1], dd.m0)));
      z = __dadd_rn(z, __dmul_rn(h, __ddiv_rn(P[2], dd.m0)));
      D.x[p] = x; D.y[p] = y; D.z[p] = z;
    }
    if (pre) {
      const double vx = D.vx[p], vy = D.vy[p], vz = D.vz[p];
      const float fx = __double2float_rn(x), fy = __double2float_rn(y), fz = __double2float_rn(z);
      D.xf[p] = fx; D.yf[p] = fy; D.zf[p] = fz;
      D.xl[p] = __double2float_rn(x - (double)fx);
      D.yl[p] = __double2float_rn(y - (double)fy);
      D.zl[p] = __double2float_rn(z - (double)fz);
      D.vxf[p] = __double2float_rn(vx); D.vyf[p] = __double2float_rn(vy); D.vzf[p] = __double2float_rn(vz);
      D.gmf[p] = __double2float_rn(D.gm[p]);
      D.lamf[p] = __double2float_ru(dd.hill_scale * D.rh[p]);
      const double sig = fmax(fmax(fabs(x), fabs(y)), fabs(z)) +
                         dd.dt * fmax(fmax(fabs(vx), fabs(vy)), fabs(vz));
      D.sigf[p] = __double2float_ru(sig);
    }
  }
}

void launch_sundrift(const Dev &D, long long npart, int pre, cudaStream_t s) {
  if (npart <= 0) return;
  long long blocks = (npart + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  k_sundrift<<<(int)blocks, 256, 0, s>>>(D, npart, pre);
}

// --------------------------------------------------------------------------------------------
// kick: a_p = fixed-order sum of the trapezoid partials that touch p, then v_p = v_p + (tau/2) a_p.
// Macro-tiles are (row quad q, column group g), C = SYM_MACRO_COLS column blocks per group, g from
// 4q / C; block B of the system has its row partials in (B/4, g), g = 4(B/4)/C..ng-1 (row slot
// B % 4), then its column partials in (q, B/C), q = 0..B/4 (column slot B % C; the diagonal
// tiles' column sides are folded into their rows).  Macro-tile (q, g) is entry
// tile_base + q ng - (4/C) q (q - 1)/2 + (g - 4q/C) of the list.
// --------------------------------------------------------------------------------------------
__device__ __forceinline__ int macro_index(const DiskDesc &dd, int ng, int q, int g) {
  return dd.tile_base + q * ng - (4 / SYM_MACRO_COLS) * ((q * (q - 1)) / 2) + (g - (4 / SYM_MACRO_COLS) * q);
}

__global__ void k_reduce(Dev D, long long npart) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < npart;
       p += (long long)gridDim.x * blockDim.x) {
    const int d = D.blk_disk[p >> 5];
    if (d < 0) continue;
    const DiskDesc &dd = D.disks[d];
    if (!dd.active) continue;
    const int li = (int)p - dd.off;
    if (li >= dd.n || !D.alive[p]) continue;
    const int B = li >> 5, lane = li & 31;
    if (B >= dd.nbm) continue;                  // a block of field particles: kicked by k_field_*
    const int C = SYM_MACRO_COLS, ng = (dd.nbm + C - 1) / C, qB = B >> 2, gB = B / C;
    const int rslot = (B & 3) * 96 + lane, cslot = 384 + (B % C) * 96 + lane;
    // the partials of p in a fixed order (its rows, then its columns); two interleaved sums
    // (even and odd terms) keep two loads in flight, combined at the end
    const int g0 = (4 / C) * qB, nrow = ng - g0;
    const int nterm = nrow + qB + 1;
    auto ptr = [&](int t) -> const double * {
      if (t < nrow) return D.part + (size_t)macro_index(dd, ng, qB, g0 + t) * SYM_MACRO_PART + rslot;
      const int q = t - nrow;
      return D.part + (size_t)macro_index(dd, ng, q, gB) * SYM_MACRO_PART + cslot;
    };
    double ax0 = 0.0, ay0 = 0.0, az0 = 0.0, ax1 = 0.0, ay1 = 0.0, az1 = 0.0;
    int t = 0;
    for (; t + 1 < nterm; t += 2) {
      const double *p0 = ptr(t), *p1 = ptr(t + 1);
      ax0 += p0[0]; ay0 += p0[32]; az0 += p0[64];
      ax1 += p1[0]; ay1 += p1[32]; az1 += p1[64];
    }
    if (t < nterm) {
      const double *p0 = ptr(t);
      ax0 += p0[0]; ay0 += p0[32]; az0 += p0[64];
    }
    const double ax = ax0 + ax1, ay = ay0 + ay1, az = az0 + az1;
    const double h = 0.5 * dd.dt;
    D.vx[p] = __dadd_rn(D.vx[p], __dmul_rn(h, ax));
    D.vy[p] = __dadd_rn(D.vy[p], __dmul_rn(h, ay));
    D.vz[p] = __dadd_rn(D.vz[p], __dmul_rn(h, az));
  }
}

// mixed precision: the partials are (sum, compensation) FP32 pairs (value = sum - comp); they
// are accumulated in FP32 with Kahan compensation and the total is carried into FP64 once.
__device__ __forceinline__ void kahan_add(float &s, float &c, float term) {
  const float y = term - c;
  const float t = s + y;
  c = (t - s) - y;
  s = t;
}

__global__ void k_reduce_mixed(Dev D, long long npart) {
  const float2 *part = reinterpret_cast<const float2 *>(D.part);
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < npart;
       p += (long long)gridDim.x * blockDim.x) {
    const int d = D.blk_disk[p >> 5];
    if (d < 0) continue;
    const DiskDesc &dd = D.disks[d];
    if (!dd.active) continue;
    const int li = (int)p - dd.off;
    if (li >= dd.n || !D.alive[p]) continue;
    const int B = li >> 5, lane = li & 31;
    if (B >= dd.nbm) continue;                  // a block of field particles: kicked by k_field_mixed
    const int C = SYM_MACRO_COLS, ng = (dd.nbm + C - 1) / C, qB = B >> 2, gB = B / C;
    const int rslot = (B & 3) * 96 + lane, cslot = 384 + (B % C) * 96 + lane;
    float s[3] = {0.f, 0.f, 0.f}, c[3] = {0.f, 0.f, 0.f};
    for (int g = (4 / C) * qB; g < ng; ++g) {
      const float2 *pp = part + (size_t)macro_index(dd, ng, qB, g) * SYM_MACRO_PART + rslot;
      for (int k = 0; k < 3; ++k) { kahan_add(s[k], c[k], pp[32 * k].x); kahan_add(s[k], c[k], -pp[32 * k].y); }
    }
    for (int q = 0; q <= qB; ++q) {
      const float2 *pp = part + (size_t)macro_index(dd, ng, q, gB) * SYM_MACRO_PART + cslot;
      for (int k = 0; k < 3; ++k) { kahan_add(s[k], c[k], pp[32 * k].x); kahan_add(s[k], c[k], -pp[32 * k].y); }
    }
    const double h = 0.5 * dd.dt;
    D.vx[p] = fma(h, (double)s[0] - (double)c[0], D.vx[p]);
    D.vy[p] = fma(h, (double)s[1] - (double)c[1], D.vy[p]);
    D.vz[p] = fma(h, (double)s[2] - (double)c[2], D.vz[p]);
  }
}

void launch_reduce(const Dev &D, long long npart, int precision, cudaStream_t s) {
  if (npart <= 0) return;
  long long blocks = (npart + 127) / 128;
  if (blocks > 8192) blocks = 8192;
  if (precision == SYMBA_PRECISION_MIXED) k_reduce_mixed<<<(int)blocks, 128, 0, s>>>(D, npart);
  else k_reduce<<<(int)blocks, 128, 0, s>>>(D, npart);
}

// two-float split of the positions before kick 2 (mixed precision)
__global__ void k_split(Dev D, long long npart) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < npart;
       p += (long long)gridDim.x * blockDim.x) {
    const double x = D.x[p], y = D.y[p], z = D.z[p];
    const float fx = __double2float_rn(x), fy = __double2float_rn(y), fz = __double2float_rn(z);
    D.xf[p] = fx; D.yf[p] = fy; D.zf[p] = fz;
    D.xl[p] = __double2float_rn(x - (double)fx);
    D.yl[p] = __double2float_rn(y - (double)fy);
    D.zl[p] = __double2float_rn(z - (double)fz);
    D.gmf[p] = __double2float_rn(D.gm[p]);
  }
}

void launch_split(const Dev &D, long long npart, cudaStream_t s) {
  if (npart <= 0) return;
  long long blocks = (npart + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  k_split<<<(int)blocks, 256, 0, s>>>(D, npart);
}

// --------------------------------------------------------------------------------------------
// Kepler drift tau (mu = G m0) of every live particle that is in no encounter group
// --------------------------------------------------------------------------------------------
__global__ void k_drift(Dev D, long long npart) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < npart;
       p += (long long)gridDim.x * blockDim.x) {
    const int d = D.blk_disk[p >> 5];
    if (d < 0) continue;
    const DiskDesc &dd = D.disks[d];
    if (!dd.active || !D.alive[p] || D.gid[p] >= 0) continue;
    if ((int)p - dd.off >= dd.n) continue;
    double x = D.x[p], y = D.y[p], z = D.z[p], vx = D.vx[p], vy = D.vy[p], vz = D.vz[p];
    const int st = kepler_drift(__dmul_rn(dd.G, dd.m0), dd.dt, x, y, z, vx, vy, vz);
    if (st != SYMBA_OK) set_status(&D.stat[d], st);
    D.x[p] = x; D.y[p] = y; D.z[p] = z;
    D.vx[p] = vx; D.vy[p] = vy; D.vz[p] = vz;
  }
}

void launch_drift(const Dev &D, long long npart, cudaStream_t s) {
  if (npart <= 0) return;
  long long blocks = (npart + 127) / 128;
  if (blocks > 8192) blocks = 8192;
  k_drift<<<(int)blocks, 128, 0, s>>>(D, npart);
}

// --------------------------------------------------------------------------------------------
// state transfer (n x 3 row-major <-> SoA)
// --------------------------------------------------------------------------------------------
__global__ void k_gather(Dev D, int d, int n, double *x, double *v, double *m, double *rad, int *alive,
                         double *rh) {
  const int off = D.disks[d].off;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int p = off + i;
    if (x) { x[3 * i] = D.x[p]; x[3 * i + 1] = D.y[p]; x[3 * i + 2] = D.z[p]; }
    if (v) { v[3 * i] = D.vx[p]; v[3 * i + 1] = D.vy[p]; v[3 * i + 2] = D.vz[p]; }
    if (m) m[i] = D.m[p];
    if (rad) rad[i] = D.rad[p];
    if (alive) alive[i] = D.alive[p];
    if (rh) rh[i] = D.rh[p];
  }
}

__global__ void k_scatter(Dev D, int d, int n, const double *x, const double *v) {
  const int off = D.disks[d].off;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int p = off + i;
    D.x[p] = x[3 * i]; D.y[p] = x[3 * i + 1]; D.z[p] = x[3 * i + 2];
    D.vx[p] = v[3 * i]; D.vy[p] = v[3 * i + 1]; D.vz[p] = v[3 * i + 2];
  }
}

void launch_gather_state(const Dev &D, int d, int n, double *x, double *v, double *m, double *rad,
                         int *alive, double *rh, cudaStream_t s) {
  k_gather<<<64, 256, 0, s>>>(D, d, n, x, v, m, rad, alive, rh);
}

void launch_scatter_state(const Dev &D, int d, int n, const double *x, const double *v,
                          cudaStream_t s) {
  k_scatter<<<64, 256, 0, s>>>(D, d, n, x, v);
}

// --------------------------------------------------------------------------------------------
// energy and angular momentum of system d, each the correctly rounded sum of its terms:
//   E = sum (0.5 m_i) |v_i|^2 - sum (G m0) m_i / |x_i| + |P|^2 / (2 m0)
//       - sum_{trapezoid pairs} (G m_i) m_j / |x_j - x_i|
//   L = sum m_i (x_i x v_i)
// Terms use the operation order written, one IEEE operation each.  acc: 4 accumulators
// (E, Lx, Ly, Lz) of SA_NDIG + 1 slots, zeroed by the caller.
// --------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_energy_particles(Dev D, int d, unsigned long long *acc) {
  const DiskDesc dd = D.disks[d];
  __shared__ unsigned long long sacc[4][SA_NDIG + 1];
  for (int k = threadIdx.x; k < 4 * (SA_NDIG + 1); k += blockDim.x) (&sacc[0][0])[k] = 0ull;
  __syncthreads();
  const double Gm0 = __dmul_rn(dd.G, dd.m0);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < dd.n; i += gridDim.x * blockDim.x) {
    const int p = dd.off + i;
    if (!D.alive[p]) continue;
    const double m = D.m[p];
    const double x = D.x[p], y = D.y[p], z = D.z[p], vx = D.vx[p], vy = D.vy[p], vz = D.vz[p];
    const double v2 = __dadd_rn(__dadd_rn(__dmul_rn(vx, vx), __dmul_rn(vy, vy)), __dmul_rn(vz, vz));
    sa_add(sacc[0], __dmul_rn(__dmul_rn(0.5, m), v2));
    const double r = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y)), __dmul_rn(z, z)));
    sa_add(sacc[0], -__ddiv_rn(__dmul_rn(Gm0, m), r));
    sa_add(sacc[1], __dmul_rn(m, __dsub_rn(__dmul_rn(y, vz), __dmul_rn(z, vy))));
    sa_add(sacc[2], __dmul_rn(m, __dsub_rn(__dmul_rn(z, vx), __dmul_rn(x, vz))));
    sa_add(sacc[3], __dmul_rn(m, __dsub_rn(__dmul_rn(x, vy), __dmul_rn(y, vx))));
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const double *P = D.P + 3 * d;
    const double P2 = __dadd_rn(__dadd_rn(__dmul_rn(P[0], P[0]), __dmul_rn(P[1], P[1])), __dmul_rn(P[2], P[2]));
    sa_add(sacc[0], __ddiv_rn(P2, __dmul_rn(2.0, dd.m0)));
  }
  __syncthreads();
  for (int k = threadIdx.x; k < 4 * (SA_NDIG + 1); k += blockDim.x) {
    const unsigned long long v = (&sacc[0][0])[k];
    if (v) atomicAdd(&acc[k], v);
  }
}

__global__ void __launch_bounds__(256) k_energy_pairs(Dev D, int d, unsigned long long *acc) {
  const DiskDesc dd = D.disks[d];
  __shared__ unsigned long long sacc[SA_NDIG + 1];
  for (int k = threadIdx.x; k < SA_NDIG + 1; k += blockDim.x) sacc[k] = 0ull;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  // every 32 x 32 tile (I, J), I <= J, of the system's macro-tiles: 4 x SYM_MACRO_COLS each
  for (int t = warp; t < 4 * SYM_MACRO_COLS * dd.ntiles; t += nwarps) {
    const int4 mt = D.tiles[dd.tile_base + t / (4 * SYM_MACRO_COLS)];
    const int u = t % (4 * SYM_MACRO_COLS);
    const int I = mt.y + u / SYM_MACRO_COLS, J = mt.z + u % SYM_MACRO_COLS;
    if (I >= mt.w || J >= mt.w || J < I) continue;
    const int li = I * 32 + lane - dd.off;
    const int p = dd.off + li;
    if (li >= dd.nm || li >= dd.n || !D.alive[p]) continue;
    const double xi = D.x[p], yi = D.y[p], zi = D.z[p];
    const double Gmi = __dmul_rn(dd.G, D.m[p]);
    for (int s = 0; s < 32; ++s) {
      const int lj = J * 32 + s - dd.off;
      if (lj <= li || lj >= dd.n) continue;
      const int q = dd.off + lj;
      if (!D.alive[q]) continue;
      const double dx = __dsub_rn(D.x[q], xi), dy = __dsub_rn(D.y[q], yi), dz = __dsub_rn(D.z[q], zi);
      const double r = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)));
      sa_add(sacc, -__ddiv_rn(__dmul_rn(Gmi, D.m[q]), r));
    }
  }
  __syncthreads();
  // O(N^2) terms over all CTAs: hand the shared accumulator this CTA's digits carried
  if (threadIdx.x == 0) sa_carry(sacc);
  __syncthreads();
  for (int k = threadIdx.x; k < SA_NDIG + 1; k += blockDim.x) {
    const unsigned long long v = sacc[k];
    if (v) atomicAdd(&acc[k], v);
  }
}

__global__ void k_energy_round(const unsigned long long *acc, double *out) {
  if (threadIdx.x < 4) out[threadIdx.x] = sa_round(acc + threadIdx.x * (SA_NDIG + 1));
}

void launch_energy(const Dev &D, int d, const LaunchCfg &L, unsigned long long *acc, cudaStream_t s) {
  k_energy_particles<<<32, 256, 0, s>>>(D, d, acc);
  k_energy_pairs<<<L.sms * 4, 256, 0, s>>>(D, d, acc);
}

void launch_energy_round(unsigned long long *acc, double *out4, cudaStream_t s) {
  k_energy_round<<<1, 32, 0, s>>>(acc, out4);
}
