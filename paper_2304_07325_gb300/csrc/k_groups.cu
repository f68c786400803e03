// Grouping of the level-0 encounter pairs (Sec. 2: GENGA-style grouping; groups are then
// integrated independently).  One CTA per system:
//   1. the pairs the fused check appended in arbitrary order are put in ascending (i, j) order
//      (counting sort by i, then each row sorted by j);
//   2. connected components by a lock-free union-find that always hooks the larger root under
//      the smaller, so every component's root is its smallest index (a unique label);
//   3. groups are numbered by ascending label; every pair gets its group, every particle its
//      group id (or -1), and every group its sorted member list and sorted pair list;
//   4. the system's groups are appended to the recursion work list.
// Everything the later kernels read is independent of the order of the atomics.
#include "internal.cuh"

__device__ int block_exscan(int *a, int n) {
  __shared__ int wsum[32];
  __shared__ int carry;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  if (tid == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < n; base += blockDim.x) {
    const int i = base + tid;
    const int v = i < n ? a[i] : 0;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
      int w = lane < nw ? wsum[lane] : 0;
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += y;
      }
      if (lane < nw) wsum[lane] = w;
    }
    __syncthreads();
    const int wpre = warp ? wsum[warp - 1] : 0;
    const int c = carry;
    if (i < n) a[i] = c + wpre + x - v;
    __syncthreads();
    if (tid == 0) carry = c + wsum[nw - 1];
    __syncthreads();
  }
  return carry;
}

__device__ __forceinline__ int uf_find(int *parent, int x) {
  for (;;) {
    const int p = __ldcg(&parent[x]);
    if (p == x) return x;
    x = p;
  }
}

__device__ __forceinline__ void uf_union(int *parent, int a, int b) {
  for (;;) {
    a = uf_find(parent, a);
    b = uf_find(parent, b);
    if (a == b) return;
    if (a > b) { const int t = a; a = b; b = t; }
    const int old = atomicCAS(&parent[b], b, a);
    if (old == b) return;
  }
}

__device__ __forceinline__ bool pair_less(int ai, int aj, int bi, int bj) {
  return ai < bi || (ai == bi && aj < bj);
}

__global__ void __launch_bounds__(1024) k_groups(Dev D) {
  const int d = blockIdx.x;
  const DiskDesc dd = D.disks[d];
  if (!dd.active) return;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int off = dd.off, npad = dd.nb * 32, pb = dd.pair_base, gb = dd.group_base;
  __shared__ int s_np, s_base;
  if (tid == 0) {
    int np = D.stat[d].npairs;
    if (np > dd.pair_cap) {
      set_status(&D.stat[d], SYMBA_E_CAPACITY);
      np = dd.pair_cap;
    }
    s_np = np;
  }
  int *cnt = D.cnt + off, *start = D.start + off, *cursor = D.cursor + off;
  int *parent = D.parent + off, *inpair = D.inpair + off, *gidx = D.gidx + off;
  for (int i = tid; i < npad; i += nt) {
    cnt[i] = 0;
    parent[i] = i;
    inpair[i] = 0;
    D.gid[off + i] = -1;
  }
  __syncthreads();
  const int np = s_np;
  for (int k = tid; k < np; k += nt) {
    const int a = D.raw_i[pb + k] - off, b = D.raw_j[pb + k] - off;
    atomicAdd(&cnt[a], 1);
    inpair[a] = 1;
    inpair[b] = 1;
  }
  __syncthreads();
  for (int i = tid; i < npad; i += nt) start[i] = cnt[i];
  __syncthreads();
  block_exscan(start, npad);
  for (int i = tid; i < npad; i += nt) cursor[i] = start[i];
  __syncthreads();
  int *tmpj = D.tmpj + pb;
  for (int k = tid; k < np; k += nt) {
    const int a = D.raw_i[pb + k] - off;
    const int pos = atomicAdd(&cursor[a], 1);
    tmpj[pos] = D.raw_j[pb + k];
  }
  __syncthreads();
  // rows in ascending j, written out as the canonical list
  for (int i = tid; i < npad; i += nt) {
    const int s0 = start[i], c = cnt[i];
    for (int a = s0 + 1; a < s0 + c; ++a) {
      const int v = tmpj[a];
      int b = a - 1;
      while (b >= s0 && tmpj[b] > v) { tmpj[b + 1] = tmpj[b]; --b; }
      tmpj[b + 1] = v;
    }
    for (int r = 0; r < c; ++r) {
      D.pi[pb + s0 + r] = off + i;
      D.pj[pb + s0 + r] = tmpj[s0 + r];
    }
  }
  __syncthreads();
  for (int q = tid; q < np; q += nt) uf_union(parent, D.pi[pb + q] - off, D.pj[pb + q] - off);
  __syncthreads();
  for (int i = tid; i < npad; i += nt) {
    const int r = inpair[i] ? uf_find(parent, i) : i;
    gidx[i] = (inpair[i] && r == i) ? 1 : 0;
    cursor[i] = r;  // label
  }
  __syncthreads();
  const int ng = block_exscan(gidx, npad);
  if (tid == 0) {
    D.stat[d].ngroups = ng;
    s_base = atomicAdd(D.rec_total, ng);
  }
  int *g_mcnt = D.g_mcnt + gb, *g_pcnt = D.g_pcnt + gb, *g_moff = D.g_moff + gb,
      *g_poff = D.g_poff + gb, *g_cur = D.g_cur + gb;
  for (int g = tid; g < ng; g += nt) { g_mcnt[g] = 0; g_pcnt[g] = 0; }
  __syncthreads();
  for (int i = tid; i < npad; i += nt) {
    if (!inpair[i]) continue;
    const int g = gidx[cursor[i]];
    D.gid[off + i] = gb + g;
    atomicAdd(&g_mcnt[g], 1);
  }
  for (int q = tid; q < np; q += nt) {
    const int g = gidx[cursor[D.pi[pb + q] - off]];
    D.gop[pb + q] = g;
    atomicAdd(&g_pcnt[g], 1);
  }
  __syncthreads();
  for (int g = tid; g < ng; g += nt) { g_moff[g] = g_mcnt[g]; g_poff[g] = g_pcnt[g]; }
  __syncthreads();
  block_exscan(g_moff, ng);
  block_exscan(g_poff, ng);
  for (int g = tid; g < ng; g += nt) g_cur[g] = g_moff[g];
  __syncthreads();
  for (int i = tid; i < npad; i += nt) {
    if (!inpair[i]) continue;
    const int g = gidx[cursor[i]];
    const int pos = atomicAdd(&g_cur[g], 1);
    D.gmem[off + pos] = off + i;
  }
  __syncthreads();
  for (int g = tid; g < ng; g += nt) g_cur[g] = g_poff[g];
  __syncthreads();
  for (int q = tid; q < np; q += nt) {
    const int g = D.gop[pb + q];
    const int pos = atomicAdd(&g_cur[g], 1);
    D.gpi[pb + pos] = D.pi[pb + q];
    D.gpj[pb + pos] = D.pj[pb + q];
  }
  __syncthreads();
  for (int g = tid; g < ng; g += nt) {
    int *mem = D.gmem + off + g_moff[g];
    const int mc = g_mcnt[g];
    for (int a = 1; a < mc; ++a) {
      const int v = mem[a];
      int b = a - 1;
      while (b >= 0 && mem[b] > v) { mem[b + 1] = mem[b]; --b; }
      mem[b + 1] = v;
    }
    int *gi = D.gpi + pb + g_poff[g], *gj = D.gpj + pb + g_poff[g];
    const int pc = g_pcnt[g];
    for (int a = 1; a < pc; ++a) {
      const int vi = gi[a], vj = gj[a];
      int b = a - 1;
      while (b >= 0 && pair_less(vi, vj, gi[b], gj[b])) { gi[b + 1] = gi[b]; gj[b + 1] = gj[b]; --b; }
      gi[b + 1] = vi;
      gj[b + 1] = vj;
    }
  }
  __syncthreads();
  // absolute offsets for the consumers; work items for the recursion
  const int base = s_base;
  for (int g = tid; g < ng; g += nt) {
    g_moff[g] += off;
    g_poff[g] += pb;
    D.rec_items[base + g] = gb + g;
  }
}

void launch_groups(const Dev &D, int ndisks, cudaStream_t s) {
  if (ndisks > 0) k_groups<<<ndisks, 1024, 0, s>>>(D);
}
