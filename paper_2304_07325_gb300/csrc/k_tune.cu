// Launch-schedule support: the order in which the persistent recursion warps take the encounter
// groups, and a fingerprint of the pool's state with which the autotuner checks that every
// schedule it tried produced the same step.
//
// Group order.  The step ends when the longest chain of dependent recursion sub-steps ends
// (Sec. 2: each group is integrated on its own), so when there are more groups than warps the
// groups with the longest chains should start first.  The chain length is estimated from the
// straight-line relative motion over the step that the level-0 check used: a pair whose closest
// approach d_min lies inside shell k (R_k = R_0 / ratio^k) sub-steps level k with h = tau / M^k,
// so it takes about M^k sub-steps for every step it stays inside, and it stays about
// 2 R_k / |dv| of the step tau.  A group's estimate is the largest over its pairs; groups are
// sorted by it, descending, ties by group slot.  Only the order changes: every group is still
// integrated by one warp from the same state, so no result depends on it.
#include "internal.cuh"

#define SYM_ORDER_CAP 16384     // groups ordered per step (shared-memory sort); more keep label order

__device__ float pair_chain_estimate(const Dev &D, const DiskDesc &dd, int i, int j) {
  const double dx = D.x[j] - D.x[i], dy = D.y[j] - D.y[i], dz = D.z[j] - D.z[i];
  const double ux = D.vx[j] - D.vx[i], uy = D.vy[j] - D.vy[i], uz = D.vz[j] - D.vz[i];
  const double r2 = dx * dx + dy * dy + dz * dz;
  const double v2 = ux * ux + uy * uy + uz * uz;
  const double vr = dx * ux + dy * uy + dz * uz;
  const double tau = dd.dt;
  double dmin2 = r2;
  if (vr < 0.0 && v2 > 0.0) {
    const double t = -vr / v2;
    dmin2 = t < tau ? r2 - vr * vr / v2 : r2 + tau * (2.0 * vr + tau * v2);
  }
  const double R0 = dd.hill_scale * (D.rh[i] + D.rh[j]);
  if (!(R0 > 0.0) || !(dmin2 < R0 * R0)) return 1.0f;
  const double dmin = sqrt(fmax(dmin2, 1e-300));
  int k = (int)ceil(log(R0 / dmin) / log(dd.shell_ratio));
  k = max(1, min(k, dd.max_depth));
  const double Rk = R0 * pow(dd.shell_ratio, -(double)k);
  const double vrel = sqrt(v2);
  const double stay = vrel > 0.0 ? fmin(1.0, 2.0 * Rk / (vrel * tau)) : 1.0;
  const double c = pow((double)dd.M, (double)k) * stay;
  return (c >= 0.0 && c < 3.0e38) ? (float)c : 3.0e38f;
}

__global__ void __launch_bounds__(1024) k_order_groups(Dev D) {
  extern __shared__ unsigned long long key[];
  const int n = *D.rec_total;
  if (n <= 1 || n > SYM_ORDER_CAP) return;
  int p2 = 1;
  while (p2 < n) p2 <<= 1;
  for (int t = threadIdx.x; t < p2; t += blockDim.x) {
    if (t < n) {
      const int slot = D.rec_items[t];
      const int p0 = D.g_poff[slot], np = D.g_pcnt[slot];
      float c = 0.0f;
      if (np > 0) {
        const DiskDesc &dd = D.disks[find_disk(D.blk_disk, D.gpi[p0])];
        for (int q = p0; q < p0 + np; ++q) c = fmaxf(c, pair_chain_estimate(D, dd, D.gpi[q], D.gpj[q]));
      }
      // ascending keys: larger estimate first (complemented bits of a non-negative float),
      // then the smaller slot
      key[t] = ((unsigned long long)(~__float_as_uint(c)) << 32) | (unsigned)slot;
    } else {
      key[t] = ~0ull;
    }
  }
  __syncthreads();
  for (int k = 2; k <= p2; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < p2; i += blockDim.x) {
        const int l = i ^ j;
        if (l > i) {
          const unsigned long long a = key[i], b = key[l];
          if ((a > b) == ((i & k) == 0)) { key[i] = b; key[l] = a; }
        }
      }
      __syncthreads();
    }
  }
  for (int t = threadIdx.x; t < n; t += blockDim.x) D.rec_items[t] = (int)(unsigned)(key[t] & 0xFFFFFFFFull);
}

bool order_groups_init() {
  return cudaFuncSetAttribute(k_order_groups, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              SYM_ORDER_CAP * (int)sizeof(unsigned long long)) == cudaSuccess;
}

void launch_order_groups(const Dev &D, cudaStream_t s) {
  k_order_groups<<<1, 1024, SYM_ORDER_CAP * sizeof(unsigned long long), s>>>(D);
}

// --------------------------------------------------------------------------------------------
// State fingerprint: a sum modulo 2^64 of a 64-bit mix of every state word with its position,
// so it does not depend on the order in which threads add their terms.
// --------------------------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void k_state_hash(Dev D, long long np, int ndisks, unsigned long long *h) {
  unsigned long long acc = 0ull;
  const double *arr[9] = {D.x, D.y, D.z, D.vx, D.vy, D.vz, D.m, D.rad, D.gm};
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < np;
       p += (long long)gridDim.x * blockDim.x) {
#pragma unroll
    for (int a = 0; a < 9; ++a)
      acc += mix64((unsigned long long)__double_as_longlong(arr[a][p]) ^ mix64((unsigned long long)(p * 16 + a)));
    acc += mix64((unsigned long long)(unsigned)D.alive[p] ^ mix64((unsigned long long)(p * 16 + 9)));
  }
  if (blockIdx.x == 0) {
    for (int d = threadIdx.x; d < ndisks; d += blockDim.x) {
      const DiskStat &s = D.stat[d];
      acc += mix64((unsigned long long)s.substeps ^ mix64(0x5000000000000000ull + 8ull * d));
      acc += mix64((unsigned long long)s.merges ^ mix64(0x5000000000000001ull + 8ull * d));
      acc += mix64((unsigned long long)(unsigned)s.npairs ^ mix64(0x5000000000000002ull + 8ull * d));
      acc += mix64((unsigned long long)(unsigned)s.ngroups ^ mix64(0x5000000000000003ull + 8ull * d));
      acc += mix64((unsigned long long)(unsigned)s.status ^ mix64(0x5000000000000004ull + 8ull * d));
      acc += mix64((unsigned long long)s.removals ^ mix64(0x5000000000000005ull + 8ull * d));
    }
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(h, acc);
}

void launch_state_hash(const Dev &D, long long np, int ndisks, unsigned long long *h, cudaStream_t s) {
  cudaMemsetAsync(h, 0, sizeof(unsigned long long), s);
  k_state_hash<<<304, 256, 0, s>>>(D, np, ndisks, h);
}
