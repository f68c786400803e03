// Host runtime and C ABI: pools of systems (a single-system context is a pool of one), device
// memory arenas sized at creation, first-fit allocation of particle and pair ranges, the
// trapezoid tile list, and the per-step launch sequence captured once into a CUDA graph.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <thread>
#include <vector>

#include "internal.cuh"
#include "ptr_class.h"

namespace {

struct Slot {
  bool active = false;
  int off = 0, n = 0, nm = 0, nb = 0, nbm = 0, ntiles = 0, nmacro = 0, pair_base = 0, pair_cap = 0;
  symba_params p{};
  long long merges_reported = 0;
};

// first-fit free list over [0, cap)
struct RangeAlloc {
  std::map<long long, long long> free_;  // start -> length
  void init(long long cap) { free_.clear(); if (cap > 0) free_[0] = cap; }
  long long alloc(long long len) {
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= len) {
        const long long s = it->first, l = it->second;
        free_.erase(it);
        if (l > len) free_[s + len] = l - len;
        return s;
      }
    }
    return -1;
  }
  void release(long long s, long long len) {
    auto it = free_.emplace(s, len).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) { it->second += nx->second; free_.erase(nx); }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) { pv->second += it->second; free_.erase(it); }
    }
  }
};

// trapezoid tiles of a system: (I, J), I <= J, over the column blocks that hold massive bodies
// (blocks of field particles only are rows of the field rectangle instead)
long long tiles_of(int nbm) { return (long long)nbm * (nbm + 1) / 2; }

// macro-tiles (row quads q of 4 blocks by column groups g of SYM_MACRO_COLS blocks, g from
// 4q / SYM_MACRO_COLS) of a system with nbm massive blocks
long long macros_of(int nbm) {
  const long long C = SYM_MACRO_COLS, nq = (nbm + 3) / 4, ng = (nbm + C - 1) / C;
  long long m = 0;
  for (long long q = 0; q < nq; ++q) m += ng - (4 / C) * q;
  return m;
}

// Macro-tiles a pool sized for max_tiles tiles over up to max_disks systems can need: a system of
// T tiles has nbm <= sqrt(2T) blocks and at most T / (4 C) + sqrt(2T) + 2 macro-tiles (checked
// for every nbm up to 20,000 in tests/test_abi.py), and each system's T is at most max_tiles.
long long macro_capacity(long long max_tiles, int max_disks) {
  const double root = std::sqrt(2.0 * (double)max_tiles);
  return max_tiles / (4 * SYM_MACRO_COLS) + (long long)max_disks * ((long long)std::ceil(root) + 2);
}

int default_pair_cap(const symba_params *p, int n) {
  if (p && p->pair_capacity > 0) return p->pair_capacity;
  return std::max(4096, 4 * n);
}

}  // namespace

struct symba_pool {
  int max_disks = 0, precision = 0;
  long long pcap = 0, tcap = 0, paircap = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int device = 0;
  Dev D{};
  LaunchCfg L{};
  std::vector<Slot> slots;
  RangeAlloc parts, pairs;
  long long tiles_used = 0;
  long long mcap = 0, macros_used = 0;       // macro-tiles: capacity and in use
  long long npart_hwm = 0;
  int ndisks = 0;
  std::vector<void *> allocs;
  unsigned long long *eacc = nullptr;
  double *eout = nullptr;
  cudaGraphExec_t gexec = nullptr;
  cudaGraph_t graph = nullptr;
  bool graph_ok = false;
  bool use_graph = true;
  // launch schedule (symba_schedule): tiles per kick work item (0 = sized from the tile count),
  // recursion CTAs per SM, group order
  int seg_override = 0;
  int rec_bpsm = 1;
  int group_order = 0;
  bool any_discard = false;   // some system has a removal distance: the step runs k_discard
};

struct symba_ctx {
  symba_pool *pool;
  int slot;
};

namespace {

#define CK(call)                                    \
  do {                                              \
    cudaError_t e_ = (call);                        \
    if (e_ != cudaSuccess) return SYMBA_E_CUDA;     \
  } while (0)

template <class T>
int dalloc(symba_pool *P, T **ptr, size_t count) {
  void *p = nullptr;
  if (count == 0) count = 1;
  if (cudaMalloc(&p, count * sizeof(T)) != cudaSuccess) return SYMBA_E_NOMEM;
  P->allocs.push_back(p);
  *ptr = (T *)p;
  return SYMBA_OK;
}

// a device array of the current device (or managed memory): used in place
bool is_device_ptr(const void *p) { return pointer_class(p) == PTR_DEVICE; }

// an array in another GPU's memory: rejected by every entry point
bool is_foreign_ptr(const void *p) { return p && pointer_class(p) == PTR_FOREIGN; }

// device copy of a caller array (or the array itself when it is already on the device)
struct Staged {
  const void *dev = nullptr;
  void *own = nullptr;
  ~Staged() { if (own) cudaFree(own); }
};

int stage_in(Staged &s, const void *src, size_t bytes, cudaStream_t st) {
  if (!src) return SYMBA_OK;
  const int cls = pointer_class(src);
  if (cls == PTR_FOREIGN) return SYMBA_E_INVAL;
  if (cls == PTR_DEVICE) { s.dev = src; return SYMBA_OK; }
  if (cudaMalloc(&s.own, bytes ? bytes : 1) != cudaSuccess) return SYMBA_E_NOMEM;
  CK(cudaMemcpyAsync(s.own, src, bytes, cudaMemcpyHostToDevice, st));
  s.dev = s.own;
  return SYMBA_OK;
}

void invalidate_graph(symba_pool *P) {
  if (P->gexec) cudaGraphExecDestroy(P->gexec);
  if (P->graph) cudaGraphDestroy(P->graph);
  P->gexec = nullptr;
  P->graph = nullptr;
  P->graph_ok = false;
}

// rebuild the tile list and the per-system descriptors after an admission or eviction
int rebuild(symba_pool *P) {
  std::vector<int4> tiles;
  tiles.reserve((size_t)P->tiles_used);
  int hw = 0;
  long long phw = 0;
  for (int d = 0; d < P->max_disks; ++d) {
    Slot &s = P->slots[d];
    if (!s.active) continue;
    hw = d + 1;
    phw = std::max(phw, (long long)s.off + (long long)s.nb * SYM_TILE);
  }
  std::vector<DiskDesc> descs(P->max_disks);
  std::vector<int2> fblk;
  bool any_discard = false;
  for (int d = 0; d < P->max_disks; ++d) {
    Slot &s = P->slots[d];
    DiskDesc &dd = descs[d];
    memset(&dd, 0, sizeof(dd));
    if (!s.active) continue;
    dd.off = s.off; dd.n = s.n; dd.nm = s.nm; dd.nb = s.nb; dd.nbm = s.nbm;
    dd.tile_base = (int)tiles.size();
    dd.ntiles = s.nmacro;
    dd.pair_base = s.pair_base; dd.pair_cap = s.pair_cap;
    dd.group_base = s.off / 2;
    dd.active = 1;
    dd.M = s.p.M; dd.l = s.p.l; dd.max_depth = std::min(s.p.max_depth, SYM_MAX_LEVELS - 1);
    dd.max_substeps = s.p.max_substeps > 0 ? s.p.max_substeps : (1 << 22);
    dd.dt = s.p.dt; dd.shell_ratio = s.p.shell_ratio; dd.hill_scale = s.p.hill_scale;
    dd.G = s.p.G; dd.m0 = s.p.m0;
    dd.rmin2 = s.p.rmin > 0.0 ? s.p.rmin * s.p.rmin : 0.0;
    dd.rmax2 = s.p.rmax > 0.0 ? s.p.rmax * s.p.rmax : 0.0;
    any_discard = any_discard || dd.rmin2 > 0.0 || dd.rmax2 > 0.0;
    const int b0 = s.off / SYM_TILE;
    const int C = SYM_MACRO_COLS, nq = (s.nbm + 3) / 4, ng = (s.nbm + C - 1) / C;
    for (int q = 0; q < nq; ++q)
      for (int g = (4 / C) * q; g < ng; ++g) tiles.push_back(make_int4(d, b0 + 4 * q, b0 + C * g, b0 + s.nbm));
    for (int B = s.nbm; B < s.nb; ++B) fblk.push_back(make_int2(d, b0 + B));
  }
  P->ndisks = hw;
  P->npart_hwm = phw;
  P->any_discard = any_discard;
  P->D.ndisks = hw;
  P->D.ntiles_total = (int)tiles.size();
  // macro-tiles per grab: one unless there are many per CTA
  long long seg = (long long)tiles.size() / std::max(1LL, (long long)P->L.trap_blocks * 8);
  P->D.seg_len = P->seg_override > 0 ? P->seg_override : (int)std::max(1LL, std::min(4LL, seg));
  if (!tiles.empty())
    CK(cudaMemcpyAsync(P->D.tiles, tiles.data(), tiles.size() * sizeof(int4), cudaMemcpyHostToDevice, P->stream));
  P->D.nfblk = (int)fblk.size();
  if (!fblk.empty())
    CK(cudaMemcpyAsync(P->D.fblk, fblk.data(), fblk.size() * sizeof(int2), cudaMemcpyHostToDevice, P->stream));
  // ck tables are filled on the device by the set-up kernel: keep them across uploads
  CK(cudaStreamSynchronize(P->stream));
  std::vector<DiskDesc> cur(P->max_disks);
  CK(cudaMemcpy(cur.data(), P->D.disks, sizeof(DiskDesc) * P->max_disks, cudaMemcpyDeviceToHost));
  for (int d = 0; d < P->max_disks; ++d) {
    memcpy(descs[d].ck, cur[d].ck, sizeof(descs[d].ck));
    memcpy(descs[d].ck2, cur[d].ck2, sizeof(descs[d].ck2));
    memcpy(descs[d].invdc, cur[d].invdc, sizeof(descs[d].invdc));
  }
  CK(cudaMemcpyAsync(P->D.disks, descs.data(), sizeof(DiskDesc) * P->max_disks, cudaMemcpyHostToDevice, P->stream));
  invalidate_graph(P);
  return SYMBA_OK;
}

// One step of every system; rec0/rec1 (optional) are recorded around the group recursion.
void enqueue_step(symba_pool *P, cudaEvent_t rec0 = nullptr, cudaEvent_t rec1 = nullptr) {
  const Dev &D = P->D;
  const long long np = P->npart_hwm;
  launch_prologue(D, P->ndisks, P->stream);
  launch_sundrift(D, np, 1, P->stream);
  launch_trap(D, P->L, 1, P->precision, P->stream);
  launch_field(D, 1, P->precision, P->stream);
  launch_reduce(D, np, P->precision, P->stream);
  launch_groups(D, P->ndisks, P->stream);
  if (P->group_order) launch_order_groups(D, P->stream);
  launch_drift(D, np, P->stream);
  if (rec0) cudaEventRecord(rec0, P->stream);
  launch_recursion(D, P->L, P->stream);
  if (rec1) cudaEventRecord(rec1, P->stream);
  if (P->precision == SYMBA_PRECISION_MIXED) launch_split(D, np, P->stream);
  launch_trap(D, P->L, 2, P->precision, P->stream);
  launch_field(D, 2, P->precision, P->stream);
  launch_reduce(D, np, P->precision, P->stream);
  if (P->any_discard) launch_discard(D, np, P->stream);
  launch_momentum(D, P->ndisks, P->stream);
  launch_sundrift(D, np, 0, P->stream);
}

__global__ void k_reset_call(DiskStat *st, int nd) {
  for (int d = threadIdx.x; d < nd; d += blockDim.x) {
    st[d].max_depth = 0;
    st[d].substeps = 0;
    st[d].max_chain = 0;
    st[d].pair_substeps = 0;
  }
}

int pool_profile(symba_pool *P, int nsteps, double *phase_ms) {
  if (nsteps < 0 || !phase_ms) return SYMBA_E_INVAL;
  for (int k = 0; k < SYMBA_NPHASES; ++k) phase_ms[k] = 0.0;
  if (nsteps == 0 || P->ndisks == 0) return SYMBA_OK;
  CK(cudaSetDevice(P->device));
  cudaEvent_t ev[SYMBA_NPHASES + 1];
  for (int k = 0; k <= SYMBA_NPHASES; ++k) CK(cudaEventCreate(&ev[k]));
  k_reset_call<<<1, 256, 0, P->stream>>>(P->D.stat, P->ndisks);
  const Dev &D = P->D;
  const long long np = P->npart_hwm;
  cudaStream_t s = P->stream;
  int rc = SYMBA_OK;
  for (int step = 0; step < nsteps && rc == SYMBA_OK; ++step) {
    cudaEventRecord(ev[0], s);
    launch_prologue(D, P->ndisks, s);
    launch_sundrift(D, np, 1, s);
    cudaEventRecord(ev[1], s);
    launch_trap(D, P->L, 1, P->precision, s);
    launch_field(D, 1, P->precision, s);
    cudaEventRecord(ev[2], s);
    launch_reduce(D, np, P->precision, s);
    cudaEventRecord(ev[3], s);
    launch_groups(D, P->ndisks, s);
    if (P->group_order) launch_order_groups(D, s);
    cudaEventRecord(ev[4], s);
    launch_drift(D, np, s);
    cudaEventRecord(ev[5], s);
    launch_recursion(D, P->L, s);
    if (P->precision == SYMBA_PRECISION_MIXED) launch_split(D, np, s);
    cudaEventRecord(ev[6], s);
    launch_trap(D, P->L, 2, P->precision, s);
    launch_field(D, 2, P->precision, s);
    cudaEventRecord(ev[7], s);
    launch_reduce(D, np, P->precision, s);
    if (P->any_discard) launch_discard(D, np, s);
    cudaEventRecord(ev[8], s);
    launch_momentum(D, P->ndisks, s);
    cudaEventRecord(ev[9], s);
    launch_sundrift(D, np, 0, s);
    cudaEventRecord(ev[10], s);
    if (cudaEventSynchronize(ev[10]) != cudaSuccess) { rc = SYMBA_E_CUDA; break; }
    for (int k = 0; k < SYMBA_NPHASES; ++k) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, ev[k], ev[k + 1]);
      phase_ms[k] += ms;
    }
  }
  for (int k = 0; k <= SYMBA_NPHASES; ++k) cudaEventDestroy(ev[k]);
  if (cudaGetLastError() != cudaSuccess) return SYMBA_E_CUDA;
  return rc;
}

int pool_step(symba_pool *P, int nsteps) {
  if (nsteps < 0) return SYMBA_E_INVAL;
  if (nsteps == 0 || P->ndisks == 0) return SYMBA_OK;
  CK(cudaSetDevice(P->device));
  k_reset_call<<<1, 256, 0, P->stream>>>(P->D.stat, P->ndisks);
  if (P->use_graph && !P->graph_ok) {
    cudaStreamCaptureStatus cs;
    CK(cudaStreamIsCapturing(P->stream, &cs));
    if (cs == cudaStreamCaptureStatusNone) {
      CK(cudaStreamBeginCapture(P->stream, cudaStreamCaptureModeThreadLocal));
      enqueue_step(P);
      cudaGraph_t g = nullptr;
      CK(cudaStreamEndCapture(P->stream, &g));
      cudaGraphExec_t ge = nullptr;
      if (cudaGraphInstantiate(&ge, g, 0) != cudaSuccess) {
        cudaGraphDestroy(g);
        return SYMBA_E_CUDA;
      }
      P->graph = g;
      P->gexec = ge;
      P->graph_ok = true;
    }
  }
  for (int s = 0; s < nsteps; ++s) {
    if (P->graph_ok) CK(cudaGraphLaunch(P->gexec, P->stream));
    else enqueue_step(P);
  }
  CK(cudaGetLastError());
  return SYMBA_OK;
}

int pool_create(symba_pool **out, int max_disks, long long max_particles, long long max_tiles,
                long long pair_total, int precision, void *stream) {
  if (!out || max_disks < 1 || max_particles < 1 || max_tiles < 1) return SYMBA_E_INVAL;
  if (precision != SYMBA_PRECISION_FP64 && precision != SYMBA_PRECISION_MIXED) return SYMBA_E_INVAL;
  symba_pool *P = new symba_pool();
  *out = nullptr;
  CK(cudaGetDevice(&P->device));
  P->max_disks = max_disks;
  P->precision = precision;
  P->pcap = ((max_particles + SYM_TILE - 1) / SYM_TILE) * SYM_TILE + (long long)SYM_TILE * max_disks;
  P->tcap = max_tiles;
  P->mcap = macro_capacity(max_tiles, max_disks);
  P->paircap = pair_total;
  if (stream) P->stream = (cudaStream_t)stream;
  else {
    if (cudaStreamCreateWithFlags(&P->stream, cudaStreamNonBlocking) != cudaSuccess) { delete P; return SYMBA_E_CUDA; }
    P->own_stream = true;
  }
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, P->device) != cudaSuccess) { delete P; return SYMBA_E_CUDA; }
  P->L.sms = prop.multiProcessorCount;
  P->L.trap_blocks = P->L.sms * trap_blocks_per_sm(precision);
  P->L.rec_blocks = P->L.sms * recursion_blocks_per_sm();
  if (!order_groups_init()) {
    if (P->own_stream) cudaStreamDestroy(P->stream);
    delete P;
    return SYMBA_E_CUDA;
  }
  const long long n = P->pcap, pc = P->paircap, gs = n / 2 + 1;
  Dev &D = P->D;
  int st = SYMBA_OK;
  auto A = [&](auto **ptr, size_t cnt) { if (st == SYMBA_OK) st = dalloc(P, ptr, cnt); };
  A(&D.x, n); A(&D.y, n); A(&D.z, n); A(&D.vx, n); A(&D.vy, n); A(&D.vz, n);
  A(&D.m, n); A(&D.gm, n); A(&D.rad, n); A(&D.rh, n);
  A(&D.alive, n); A(&D.gid, n);
  A(&D.xf, n); A(&D.yf, n); A(&D.zf, n); A(&D.vxf, n); A(&D.vyf, n); A(&D.vzf, n);
  A(&D.lamf, n); A(&D.sigf, n); A(&D.xl, n); A(&D.yl, n); A(&D.zl, n); A(&D.gmf, n);
  A(&D.blk_disk, n / SYM_TILE + 1);
  A(&D.disks, max_disks); A(&D.stat, max_disks); A(&D.P, 3 * max_disks);
  A(&D.sacc, (size_t)max_disks * 3 * (SA_NDIG + 1));
  A(&D.tiles, P->mcap);
  A(&D.fblk, n / SYM_TILE + 1);
  A(&D.part, (size_t)P->mcap * SYM_MACRO_PART);
  A(&D.work, 4);
  A(&D.raw_i, pc); A(&D.raw_j, pc); A(&D.pi, pc); A(&D.pj, pc); A(&D.gop, pc);
  A(&D.gpi, pc); A(&D.gpj, pc); A(&D.lev, pc); A(&D.tmpj, pc);
  A(&D.perm, pc); A(&D.ptmp, pc); A(&D.pR0, pc); A(&D.pinvR0, pc);
  A(&D.mperm, n); A(&D.mtmp, n);
  A(&D.gx, n); A(&D.gy, n); A(&D.gz, n); A(&D.gvx, n); A(&D.gvy, n); A(&D.gvz, n);
  A(&D.gmm, n); A(&D.ggm, n); A(&D.grad, n); A(&D.grh, n); A(&D.galive, n);
  A(&D.gpa, pc); A(&D.gpb, pc);
  A(&D.pf, 5 * pc); A(&D.adj, 2 * pc);
  A(&D.cnt, n); A(&D.start, n); A(&D.cursor, n); A(&D.parent, n); A(&D.inpair, n);
  A(&D.gidx, n); A(&D.mslot, n); A(&D.adj_off, n); A(&D.adj_cnt, n);
  A(&D.acc, 3 * n);
  A(&D.g_moff, gs); A(&D.g_mcnt, gs); A(&D.g_poff, gs); A(&D.g_pcnt, gs); A(&D.g_cur, gs);
  A(&D.gmem, n); A(&D.rec_items, gs); A(&D.rec_total, 1);
  A(&D.lcache, (size_t)P->L.sms * SYM_REC_BPSM_MAX * 4 * SYM_PAIR_LC);   // any schedule
  A(&P->eacc, 4 * (SA_NDIG + 1)); A(&P->eout, 4);
  if (st != SYMBA_OK) { symba_pool_free(P); return st; }
  if (cudaMemsetAsync(D.blk_disk, 0xFF, sizeof(int) * (n / SYM_TILE + 1), P->stream) != cudaSuccess ||
      cudaMemsetAsync(D.disks, 0, sizeof(DiskDesc) * max_disks, P->stream) != cudaSuccess ||
      cudaMemsetAsync(D.stat, 0, sizeof(DiskStat) * max_disks, P->stream) != cudaSuccess ||
      cudaMemsetAsync(D.work, 0, sizeof(int) * 4, P->stream) != cudaSuccess ||
      cudaMemsetAsync(D.sacc, 0, sizeof(unsigned long long) * max_disks * 3 * (SA_NDIG + 1), P->stream) != cudaSuccess ||
      cudaMemsetAsync(D.rec_total, 0, sizeof(int), P->stream) != cudaSuccess ||
      cudaMemsetAsync(D.alive, 0, sizeof(int) * n, P->stream) != cudaSuccess) {
    symba_pool_free(P);
    return SYMBA_E_CUDA;
  }
  P->slots.assign(max_disks, Slot());
  P->parts.init(n);
  P->pairs.init(pc);
  *out = P;
  return SYMBA_OK;
}

int pool_admit(symba_pool *P, const symba_params *p, int n, int nm, const double *x, const double *v,
               const double *m, const double *radius, const double *rhill, int *slot) {
  if (!P || !p || !x || !v || !m || !radius || n < 1 || nm < 0 || nm > n) return SYMBA_E_INVAL;
  if (p->dt == 0.0 || !(p->shell_ratio > 1.0) || p->M < 1 || p->l < 1 || p->max_depth < 1 ||
      !(p->m0 > 0.0) || !(p->hill_scale >= 0.0) || !(p->rmin >= 0.0) || !(p->rmax >= 0.0) ||
      !std::isfinite(p->rmin) || !std::isfinite(p->rmax) || (p->rmax > 0.0 && p->rmin >= p->rmax))
    return SYMBA_E_INVAL;
  CK(cudaSetDevice(P->device));
  int d = -1;
  for (int k = 0; k < P->max_disks; ++k) if (!P->slots[k].active) { d = k; break; }
  if (d < 0) return SYMBA_E_NOMEM;
  Slot s;
  s.n = n; s.nm = nm; s.p = *p;
  s.nb = (n + SYM_TILE - 1) / SYM_TILE;
  s.nbm = (nm + SYM_TILE - 1) / SYM_TILE;
  s.ntiles = (int)tiles_of(s.nbm);
  s.nmacro = (int)macros_of(s.nbm);
  s.pair_cap = default_pair_cap(p, n);
  if (P->tiles_used + s.ntiles > P->tcap || P->macros_used + s.nmacro > P->mcap) return SYMBA_E_NOMEM;
  const long long po = P->parts.alloc((long long)s.nb * SYM_TILE);
  if (po < 0) return SYMBA_E_NOMEM;
  const long long pb = P->pairs.alloc(s.pair_cap);
  if (pb < 0) { P->parts.release(po, (long long)s.nb * SYM_TILE); return SYMBA_E_NOMEM; }
  s.off = (int)po;
  s.pair_base = (int)pb;
  s.active = true;
  P->slots[d] = s;
  P->tiles_used += s.ntiles;
  P->macros_used += s.nmacro;
  // block -> system map
  std::vector<int> bd(s.nb, d);
  CK(cudaMemcpyAsync(P->D.blk_disk + s.off / SYM_TILE, bd.data(), sizeof(int) * s.nb, cudaMemcpyHostToDevice, P->stream));
  int st = rebuild(P);
  if (st != SYMBA_OK) return st;
  launch_setup_disk(P->D, d, P->stream);
  Staged sx, sv, sm, sr, sh;
  if ((st = stage_in(sx, x, sizeof(double) * 3 * n, P->stream)) != SYMBA_OK) return st;
  if ((st = stage_in(sv, v, sizeof(double) * 3 * n, P->stream)) != SYMBA_OK) return st;
  if ((st = stage_in(sm, m, sizeof(double) * n, P->stream)) != SYMBA_OK) return st;
  if ((st = stage_in(sr, radius, sizeof(double) * n, P->stream)) != SYMBA_OK) return st;
  if ((st = stage_in(sh, rhill, sizeof(double) * n, P->stream)) != SYMBA_OK) return st;
  launch_init_state(P->D, d, n, (const double *)sx.dev, (const double *)sv.dev, (const double *)sm.dev,
                    (const double *)sr.dev, (const double *)sh.dev, rhill == nullptr ? 1 : 0, P->stream);
  launch_momentum(P->D, P->ndisks, P->stream);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(P->stream));  // staging buffers are freed on return
  if (slot) *slot = d;
  return SYMBA_OK;
}

int read_stat(symba_pool *P, int d, DiskStat *out) {
  CK(cudaStreamSynchronize(P->stream));
  CK(cudaMemcpy(out, P->D.stat + d, sizeof(DiskStat), cudaMemcpyDeviceToHost));
  return SYMBA_OK;
}

int slot_status(symba_pool *P, int d) {
  DiskStat st;
  int r = read_stat(P, d, &st);
  if (r != SYMBA_OK) return r;
  if (st.status != 0) return st.status;
  Slot &s = P->slots[d];
  if ((long long)st.merges > s.merges_reported) {
    s.merges_reported = (long long)st.merges;
    return SYMBA_COLLISION;
  }
  return SYMBA_OK;
}

bool valid_slot(symba_pool *P, int d) { return P && d >= 0 && d < P->max_disks && P->slots[d].active; }

int get_state(symba_pool *P, int d, double *x, double *v, double *m, double *rad, int *alive) {
  if (!valid_slot(P, d)) return SYMBA_E_INVAL;
  CK(cudaSetDevice(P->device));
  const int n = P->slots[d].n;
  if (is_foreign_ptr(x) || is_foreign_ptr(v) || is_foreign_ptr(m) || is_foreign_ptr(rad) || is_foreign_ptr(alive))
    return SYMBA_E_INVAL;
  double *dx = nullptr, *dv = nullptr, *dm = nullptr, *dr = nullptr;
  int *da = nullptr;
  const bool hx = x && !is_device_ptr(x), hv = v && !is_device_ptr(v), hm = m && !is_device_ptr(m),
             hr = rad && !is_device_ptr(rad), ha = alive && !is_device_ptr(alive);
  int st = SYMBA_OK;
  auto tmp = [&](bool need, void **pp, size_t bytes) {
    if (need && st == SYMBA_OK && cudaMalloc(pp, bytes) != cudaSuccess) st = SYMBA_E_NOMEM;
  };
  tmp(hx, (void **)&dx, sizeof(double) * 3 * n);
  tmp(hv, (void **)&dv, sizeof(double) * 3 * n);
  tmp(hm, (void **)&dm, sizeof(double) * n);
  tmp(hr, (void **)&dr, sizeof(double) * n);
  tmp(ha, (void **)&da, sizeof(int) * n);
  if (st == SYMBA_OK) {
    launch_gather_state(P->D, d, n, hx ? dx : x, hv ? dv : v, hm ? dm : m, hr ? dr : rad, ha ? da : alive,
                        nullptr, P->stream);
    if (hx) cudaMemcpyAsync(x, dx, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, P->stream);
    if (hv) cudaMemcpyAsync(v, dv, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, P->stream);
    if (hm) cudaMemcpyAsync(m, dm, sizeof(double) * n, cudaMemcpyDeviceToHost, P->stream);
    if (hr) cudaMemcpyAsync(rad, dr, sizeof(double) * n, cudaMemcpyDeviceToHost, P->stream);
    if (ha) cudaMemcpyAsync(alive, da, sizeof(int) * n, cudaMemcpyDeviceToHost, P->stream);
    if (cudaStreamSynchronize(P->stream) != cudaSuccess) st = SYMBA_E_CUDA;
  }
  cudaFree(dx); cudaFree(dv); cudaFree(dm); cudaFree(dr); cudaFree(da);
  if (st != SYMBA_OK) return st;
  return slot_status(P, d);
}

int get_rhill(symba_pool *P, int d, double *rh) {
  if (!valid_slot(P, d) || !rh) return SYMBA_E_INVAL;
  CK(cudaSetDevice(P->device));
  const int n = P->slots[d].n;
  if (is_foreign_ptr(rh)) return SYMBA_E_INVAL;
  const bool host = !is_device_ptr(rh);
  double *dh = nullptr;
  if (host && cudaMalloc(&dh, sizeof(double) * n) != cudaSuccess) return SYMBA_E_NOMEM;
  launch_gather_state(P->D, d, n, nullptr, nullptr, nullptr, nullptr, nullptr, host ? dh : rh, P->stream);
  if (host) cudaMemcpyAsync(rh, dh, sizeof(double) * n, cudaMemcpyDeviceToHost, P->stream);
  const cudaError_t e = cudaStreamSynchronize(P->stream);
  cudaFree(dh);
  if (e != cudaSuccess) return SYMBA_E_CUDA;
  return slot_status(P, d);
}

int set_state(symba_pool *P, int d, const double *x, const double *v) {
  if (!valid_slot(P, d) || !x || !v) return SYMBA_E_INVAL;
  CK(cudaSetDevice(P->device));
  const int n = P->slots[d].n;
  Staged sx, sv;
  int st;
  if ((st = stage_in(sx, x, sizeof(double) * 3 * n, P->stream)) != SYMBA_OK) return st;
  if ((st = stage_in(sv, v, sizeof(double) * 3 * n, P->stream)) != SYMBA_OK) return st;
  launch_scatter_state(P->D, d, n, (const double *)sx.dev, (const double *)sv.dev, P->stream);
  launch_momentum(P->D, P->ndisks, P->stream);
  CK(cudaMemsetAsync(&P->D.stat[d].status, 0, sizeof(int), P->stream));
  CK(cudaGetLastError());
  if (sx.own || sv.own) CK(cudaStreamSynchronize(P->stream));
  return SYMBA_OK;
}

int energy(symba_pool *P, int d, double *E, double *L) {
  if (!valid_slot(P, d) || !E) return SYMBA_E_INVAL;
  CK(cudaSetDevice(P->device));
  CK(cudaMemsetAsync(P->eacc, 0, sizeof(unsigned long long) * 4 * (SA_NDIG + 1), P->stream));
  launch_energy(P->D, d, P->L, P->eacc, P->stream);
  launch_energy_round(P->eacc, P->eout, P->stream);
  double out[4];
  CK(cudaMemcpyAsync(out, P->eout, sizeof(out), cudaMemcpyDeviceToHost, P->stream));
  CK(cudaStreamSynchronize(P->stream));
  *E = out[0];
  if (L) { L[0] = out[1]; L[1] = out[2]; L[2] = out[3]; }
  return slot_status(P, d);
}

__global__ void k_pairs_out(Dev D, int d, int cap, int *pairs, int *gop) {
  const DiskDesc dd = D.disks[d];
  int np = D.stat[d].npairs;
  if (np > dd.pair_cap) np = dd.pair_cap;
  const int lim = np < cap ? np : cap;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < lim; q += gridDim.x * blockDim.x) {
    if (pairs) {
      pairs[2 * q] = D.pi[dd.pair_base + q] - dd.off;
      pairs[2 * q + 1] = D.pj[dd.pair_base + q] - dd.off;
    }
    if (gop) gop[q] = D.gop[dd.pair_base + q];
  }
}

int enc_groups(symba_pool *P, int d, int *pairs, int *gop, int cap, int *npairs, int *ngroups) {
  if (!valid_slot(P, d) || cap < 0) return SYMBA_E_INVAL;
  CK(cudaSetDevice(P->device));
  if (is_foreign_ptr(pairs) || is_foreign_ptr(gop)) return SYMBA_E_INVAL;
  DiskStat st;
  int r = read_stat(P, d, &st);
  if (r != SYMBA_OK) return r;
  if (npairs) *npairs = st.npairs;
  if (ngroups) *ngroups = st.ngroups;
  const int lim = std::min(std::min(st.npairs, P->slots[d].pair_cap), cap);
  if (lim > 0 && (pairs || gop)) {
    const bool hp = pairs && !is_device_ptr(pairs), hg = gop && !is_device_ptr(gop);
    int *dp = nullptr, *dg = nullptr;
    if (hp && cudaMalloc(&dp, sizeof(int) * 2 * lim) != cudaSuccess) return SYMBA_E_NOMEM;
    if (hg && cudaMalloc(&dg, sizeof(int) * lim) != cudaSuccess) { cudaFree(dp); return SYMBA_E_NOMEM; }
    k_pairs_out<<<64, 256, 0, P->stream>>>(P->D, d, lim, hp ? dp : pairs, hg ? dg : gop);
    if (hp) cudaMemcpyAsync(pairs, dp, sizeof(int) * 2 * lim, cudaMemcpyDeviceToHost, P->stream);
    if (hg) cudaMemcpyAsync(gop, dg, sizeof(int) * lim, cudaMemcpyDeviceToHost, P->stream);
    cudaError_t e = cudaStreamSynchronize(P->stream);
    cudaFree(dp);
    cudaFree(dg);
    if (e != cudaSuccess) return SYMBA_E_CUDA;
  }
  return slot_status(P, d);
}

int get_stats(symba_pool *P, int d, symba_stats *out) {
  if (!valid_slot(P, d) || !out) return SYMBA_E_INVAL;
  CK(cudaSetDevice(P->device));
  DiskStat st;
  int r = read_stat(P, d, &st);
  if (r != SYMBA_OK) return r;
  out->n_pairs = st.npairs;
  out->n_groups = st.ngroups;
  out->max_depth = st.max_depth;
  out->status = st.status;
  out->merges = (long long)st.merges;
  out->substeps = (long long)st.substeps;
  out->max_chain = (long long)st.max_chain;
  out->pair_substeps = (long long)st.pair_substeps;
  out->removals = (long long)st.removals;
  out->steps = 0;
  return SYMBA_OK;
}


// --------------------------------------------------------------------------------------------
// launch schedules and their autotuner
// --------------------------------------------------------------------------------------------
void get_schedule(const symba_pool *P, symba_schedule *s) {
  s->kick_blocks_per_sm = P->L.trap_blocks / P->L.sms;
  s->kick_tiles_per_item = P->D.seg_len;
  s->rec_blocks_per_sm = P->rec_bpsm;
  s->group_order = P->group_order;
}

bool schedule_valid(const symba_pool *P, const symba_schedule *s) {
  return s->kick_blocks_per_sm >= 1 && s->kick_blocks_per_sm <= trap_blocks_per_sm(P->precision) &&
         s->kick_tiles_per_item >= 1 && s->kick_tiles_per_item <= 64 && s->rec_blocks_per_sm >= 1 &&
         s->rec_blocks_per_sm <= SYM_REC_BPSM_MAX && (s->group_order == 0 || s->group_order == 1);
}

void apply_schedule(symba_pool *P, const symba_schedule *s) {
  P->L.trap_blocks = P->L.sms * s->kick_blocks_per_sm;
  P->seg_override = s->kick_tiles_per_item;
  P->D.seg_len = s->kick_tiles_per_item;
  P->rec_bpsm = s->rec_blocks_per_sm;
  P->L.rec_blocks = P->L.sms * s->rec_blocks_per_sm;
  P->group_order = s->group_order;
  invalidate_graph(P);
}

// The device state a step reads and writes (everything else is per-step scratch or constant).
struct Span {
  void *p;
  size_t bytes;
};
std::vector<Span> state_spans(const symba_pool *P) {
  const Dev &D = P->D;
  const size_t n = (size_t)P->npart_hwm, nd = (size_t)P->max_disks;
  std::vector<Span> v;
  for (double *a : {D.x, D.y, D.z, D.vx, D.vy, D.vz, D.m, D.gm, D.rad, D.rh}) v.push_back({a, n * sizeof(double)});
  for (int *a : {D.alive, D.gid}) v.push_back({a, n * sizeof(int)});
  for (float *a : {D.xf, D.yf, D.zf, D.vxf, D.vyf, D.vzf, D.lamf, D.sigf, D.xl, D.yl, D.zl, D.gmf})
    v.push_back({a, n * sizeof(float)});
  v.push_back({D.P, 3 * nd * sizeof(double)});
  v.push_back({D.sacc, nd * 3 * (SA_NDIG + 1) * sizeof(unsigned long long)});
  v.push_back({D.stat, nd * sizeof(DiskStat)});
  return v;
}

size_t span_slot(size_t bytes) { return (bytes + 255) & ~(size_t)255; }

int copy_spans(const std::vector<Span> &v, char *buf, bool save, cudaStream_t s) {
  size_t off = 0;
  for (const Span &sp : v) {
    if (sp.bytes) {
      if (save) CK(cudaMemcpyAsync(buf + off, sp.p, sp.bytes, cudaMemcpyDeviceToDevice, s));
      else CK(cudaMemcpyAsync(sp.p, buf + off, sp.bytes, cudaMemcpyDeviceToDevice, s));
    }
    off += span_slot(sp.bytes);
  }
  return SYMBA_OK;
}

int pool_autotune(symba_pool *P, int reps, symba_tune_result *out) {
  if (reps < 1) return SYMBA_E_INVAL;
  CK(cudaSetDevice(P->device));
  symba_tune_result r;
  memset(&r, 0, sizeof(r));
  get_schedule(P, &r.chosen);
  r.identical = 1;
  bool any = false;
  for (int d = 0; d < P->max_disks; ++d) any = any || P->slots[d].active;
  if (!any || P->ndisks == 0 || P->D.ntiles_total <= 0) {
    if (out) *out = r;
    return SYMBA_OK;
  }
  CK(cudaStreamSynchronize(P->stream));
  const symba_schedule before = r.chosen;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  char *snap = nullptr;
  unsigned long long *hbuf = nullptr;
  int rc = SYMBA_OK;
  auto fail = [&](int code) {
    if (rc == SYMBA_OK) rc = code;
  };
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) fail(SYMBA_E_CUDA);

  // kick: the second kick (per-tile partials only) under each candidate, mean of reps launches
  auto time_kick = [&](int kb, int seg) -> double {
    P->L.trap_blocks = P->L.sms * kb;
    P->D.seg_len = seg;
    double tot = 0.0;
    for (int k = 0; k < reps && rc == SYMBA_OK; ++k) {
      float ms = 0.f;
      if (cudaMemsetAsync(P->D.work + 1, 0, sizeof(int), P->stream) != cudaSuccess ||
          cudaEventRecord(e0, P->stream) != cudaSuccess) { fail(SYMBA_E_CUDA); break; }
      launch_trap(P->D, P->L, 2, P->precision, P->stream);
      if (cudaEventRecord(e1, P->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
          cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) { fail(SYMBA_E_CUDA); break; }
      tot += ms;
    }
    return tot / reps;
  };
  symba_schedule best = before;
  if (rc == SYMBA_OK) {
    r.kick_ms_before = time_kick(before.kick_blocks_per_sm, before.kick_tiles_per_item);
    r.kick_ms = r.kick_ms_before;
    const int kmax = trap_blocks_per_sm(P->precision);
    for (int kb = 1; kb <= kmax && rc == SYMBA_OK; ++kb) {
      for (int seg : {1, 2, 4, 8, 16}) {
        const double ms = time_kick(kb, seg);
        ++r.kick_candidates;
        if (rc == SYMBA_OK && ms < r.kick_ms) {
          r.kick_ms = ms;
          best.kick_blocks_per_sm = kb;
          best.kick_tiles_per_item = seg;
        }
      }
    }
  }
  apply_schedule(P, rc == SYMBA_OK ? &best : &before);

  // recursion: the same trial step from a copy of the state under each candidate
  const std::vector<Span> spans = state_spans(P);
  size_t bytes = 0;
  for (const Span &sp : spans) bytes += span_slot(sp.bytes);
  const int cand[4][2] = {{1, 0}, {1, 1}, {2, 0}, {2, 1}};
  const int nc = 1 + 4;          // the schedule in effect first, then every candidate
  if (rc == SYMBA_OK && (cudaMalloc(&snap, bytes) != cudaSuccess ||
                         cudaMalloc(&hbuf, nc * sizeof(unsigned long long)) != cudaSuccess))
    fail(SYMBA_E_NOMEM);
  bool saved = false;
  if (rc == SYMBA_OK && copy_spans(spans, snap, true, P->stream) == SYMBA_OK) saved = true;
  else fail(SYMBA_E_CUDA);
  double rec_ms[nc] = {0.0};
  for (int c = 0; c < nc && rc == SYMBA_OK; ++c) {
    symba_schedule s = best;
    if (c > 0) {
      s.rec_blocks_per_sm = cand[c - 1][0];
      s.group_order = cand[c - 1][1];
    }
    apply_schedule(P, &s);
    if (copy_spans(spans, snap, false, P->stream) != SYMBA_OK) { fail(SYMBA_E_CUDA); break; }
    enqueue_step(P, e0, e1);
    launch_state_hash(P->D, P->npart_hwm, P->ndisks, hbuf + c, P->stream);
    float ms = 0.f;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess ||
        cudaStreamSynchronize(P->stream) != cudaSuccess) { fail(SYMBA_E_CUDA); break; }
    rec_ms[c] = ms;
    if (c > 0) ++r.recursion_candidates;
  }
  if (saved && copy_spans(spans, snap, false, P->stream) != SYMBA_OK) fail(SYMBA_E_CUDA);
  if (rc == SYMBA_OK) {
    unsigned long long h[nc];
    if (cudaMemcpyAsync(h, hbuf, sizeof(h), cudaMemcpyDeviceToHost, P->stream) != cudaSuccess ||
        cudaStreamSynchronize(P->stream) != cudaSuccess) {
      fail(SYMBA_E_CUDA);
    } else {
      for (int c = 1; c < nc; ++c) r.identical = r.identical && h[c] == h[0];
      r.recursion_ms_before = rec_ms[0];
      r.recursion_ms = rec_ms[0];
      for (int c = 1; c < nc; ++c) {
        if (rec_ms[c] < r.recursion_ms) {
          r.recursion_ms = rec_ms[c];
          best.rec_blocks_per_sm = cand[c - 1][0];
          best.group_order = cand[c - 1][1];
        }
      }
      if (best.rec_blocks_per_sm == before.rec_blocks_per_sm && best.group_order == before.group_order)
        r.recursion_ms = rec_ms[0];
    }
  }
  apply_schedule(P, rc == SYMBA_OK ? &best : &before);
  if (snap) cudaFree(snap);
  if (hbuf) cudaFree(hbuf);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (rc == SYMBA_OK) get_schedule(P, &r.chosen);
  if (out) *out = r;
  return rc;
}

}  // namespace

// ============================================================================================
// C ABI
// ============================================================================================
extern "C" {

void symba_default_params(symba_params *p) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  p->dt = 0.5;
  p->shell_ratio = 2.08;
  p->hill_scale = 6.5;
  p->G = 4.0 * M_PI * M_PI;
  p->m0 = 1.0;
  p->M = 4;
  p->l = 3;
  p->max_depth = 20;
  p->precision = SYMBA_PRECISION_FP64;
  p->pair_capacity = 0;
  p->max_substeps = 0;
}

const char *symba_status_string(int s) {
  switch (s) {
    case SYMBA_OK: return "ok";
    case SYMBA_COLLISION: return "bodies merged";
    case SYMBA_E_INVAL: return "invalid argument";
    case SYMBA_E_NOMEM: return "out of device memory or pool capacity";
    case SYMBA_E_CUDA: return "CUDA runtime error";
    case SYMBA_E_KEPLER: return "Kepler's equation did not converge";
    case SYMBA_E_DEPTH: return "recursion deeper than max_depth or sub-step budget exhausted";
    case SYMBA_E_CAPACITY: return "encounter pair list overflow";
    case SYMBA_E_NONFINITE: return "non-finite state";
    default: return "unknown status";
  }
}

long long symba_pool_footprint(int n, int n_massive, const symba_params *p) {
  if (n < 1 || n_massive < 0 || n_massive > n) return -1;
  const long long nb = (n + SYM_TILE - 1) / SYM_TILE, nbm = (n_massive + SYM_TILE - 1) / SYM_TILE;
  const long long np = nb * SYM_TILE;
  const long long per_particle = 20 * 8 + 3 * 4 + 12 * 4 + 12 * 4 + 3 * 8 + 6 * 4 / 2 + 4;
  const long long pairs = default_pair_cap(p, n);
  const long long per_pair = 13 * 4 + 7 * 8 + 2 * 4;
  return np * per_particle + pairs * per_pair + macros_of((int)nbm) * (16 + SYM_MACRO_PART * 8) + 8 * nb;
}

int symba_pool_create(symba_pool **out, int max_systems, long long max_particles, long long max_tiles,
                      int precision, void *cuda_stream) {
  const long long pair_total = std::max(4LL * max_particles, 4096LL) + 4096LL * max_systems;
  return pool_create(out, max_systems, max_particles, max_tiles, pair_total, precision, cuda_stream);
}

int symba_pool_admit(symba_pool *pool, const symba_params *p, int n, int n_massive, const double *x,
                     const double *v, const double *m, const double *radius, const double *rhill,
                     int *slot) {
  if (!pool || !p) return SYMBA_E_INVAL;
  if (p->precision != pool->precision) return SYMBA_E_INVAL;
  return pool_admit(pool, p, n, n_massive, x, v, m, radius, rhill, slot);
}

int symba_pool_step(symba_pool *pool, int nsteps) {
  if (!pool) return SYMBA_E_INVAL;
  return pool_step(pool, nsteps);
}

int symba_pool_get_schedule(symba_pool *pool, symba_schedule *s) {
  if (!pool || !s) return SYMBA_E_INVAL;
  get_schedule(pool, s);
  return SYMBA_OK;
}

int symba_pool_set_schedule(symba_pool *pool, const symba_schedule *s) {
  if (!pool || !s || !schedule_valid(pool, s)) return SYMBA_E_INVAL;
  apply_schedule(pool, s);
  return SYMBA_OK;
}

int symba_pool_autotune(symba_pool *pool, int reps, symba_tune_result *out) {
  if (!pool) return SYMBA_E_INVAL;
  return pool_autotune(pool, reps, out);
}

int symba_autotune(symba_ctx *c, int reps, symba_tune_result *out) {
  if (!c) return SYMBA_E_INVAL;
  return pool_autotune(c->pool, reps, out);
}

int symba_pool_sync(symba_pool *pool) {
  if (!pool) return SYMBA_E_INVAL;
  if (cudaStreamSynchronize(pool->stream) != cudaSuccess) return SYMBA_E_CUDA;
  int worst = SYMBA_OK;
  for (int d = 0; d < pool->max_disks; ++d) {
    if (!pool->slots[d].active) continue;
    const int s = slot_status(pool, d);
    if (s < 0 && (worst >= 0 || s < worst)) worst = s;
    else if (s > 0 && worst == SYMBA_OK) worst = s;
  }
  return worst;
}

int symba_pool_get_state(symba_pool *pool, int slot, double *x, double *v, double *m, double *radius,
                         int *alive) {
  return get_state(pool, slot, x, v, m, radius, alive);
}

int symba_pool_energy(symba_pool *pool, int slot, double *E, double L[3]) { return energy(pool, slot, E, L); }

int symba_pool_get_stats(symba_pool *pool, int slot, symba_stats *s) { return get_stats(pool, slot, s); }

int symba_pool_evict(symba_pool *pool, int slot) {
  if (!valid_slot(pool, slot)) return SYMBA_E_INVAL;
  if (cudaStreamSynchronize(pool->stream) != cudaSuccess) return SYMBA_E_CUDA;
  Slot &s = pool->slots[slot];
  std::vector<int> bd(s.nb, -1);
  if (cudaMemcpy(pool->D.blk_disk + s.off / SYM_TILE, bd.data(), sizeof(int) * s.nb, cudaMemcpyHostToDevice) != cudaSuccess)
    return SYMBA_E_CUDA;
  pool->parts.release(s.off, (long long)s.nb * SYM_TILE);
  pool->pairs.release(s.pair_base, s.pair_cap);
  pool->tiles_used -= s.ntiles;
  pool->macros_used -= s.nmacro;
  s = Slot();
  return rebuild(pool);
}

void symba_pool_free(symba_pool *pool) {
  if (!pool) return;
  if (pool->stream) cudaStreamSynchronize(pool->stream);
  invalidate_graph(pool);
  for (void *p : pool->allocs) cudaFree(p);
  if (pool->own_stream && pool->stream) cudaStreamDestroy(pool->stream);
  delete pool;
}

int symba_init(symba_ctx **out, const symba_params *p, int n, int n_massive, const double *x,
               const double *v, const double *m, const double *radius, const double *rhill,
               void *cuda_stream) {
  if (!out || !p || n < 1 || n_massive < 0 || n_massive > n) return SYMBA_E_INVAL;
  *out = nullptr;
  symba_pool *P = nullptr;
  const long long nb = (n + SYM_TILE - 1) / SYM_TILE, nbm = (n_massive + SYM_TILE - 1) / SYM_TILE;
  const long long tiles = std::max(1LL, tiles_of((int)nbm));
  int st = pool_create(&P, 1, n, tiles, default_pair_cap(p, n), p->precision, cuda_stream);
  if (st != SYMBA_OK) return st;
  int slot = -1;
  st = pool_admit(P, p, n, n_massive, x, v, m, radius, rhill, &slot);
  if (st != SYMBA_OK) { symba_pool_free(P); return st; }
  symba_ctx *c = new symba_ctx{P, slot};
  *out = c;
  return SYMBA_OK;
}

int symba_step(symba_ctx *c, int nsteps) {
  if (!c) return SYMBA_E_INVAL;
  return pool_step(c->pool, nsteps);
}

int symba_sync(symba_ctx *c) {
  if (!c) return SYMBA_E_INVAL;
  return slot_status(c->pool, c->slot);
}

int symba_step_many(symba_ctx *const *ctxs, int n, int nsteps) {
  if (!ctxs || n < 0 || nsteps < 0) return SYMBA_E_INVAL;
  for (int i = 0; i < n; ++i)
    if (!ctxs[i]) return SYMBA_E_INVAL;
  if (n == 0 || nsteps == 0) return SYMBA_OK;
  // one step in flight per context: each context's next step is launched as soon as its last
  // one has completed, so every stream stays one step deep and no system waits behind another
  std::vector<cudaEvent_t> ev((size_t)n, nullptr);
  std::vector<int> left((size_t)n, nsteps);
  std::vector<char> busy((size_t)n, 0);
  int rc = SYMBA_OK;
  for (int i = 0; i < n && rc == SYMBA_OK; ++i) {
    if (cudaSetDevice(ctxs[i]->pool->device) != cudaSuccess ||
        cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming) != cudaSuccess)
      rc = SYMBA_E_CUDA;
  }
  bool pending = true;
  while (rc == SYMBA_OK && pending) {
    bool progressed = false;
    pending = false;
    for (int i = 0; i < n && rc == SYMBA_OK; ++i) {
      if (busy[i]) {
        const cudaError_t q = cudaEventQuery(ev[i]);
        if (q == cudaSuccess) {
          busy[i] = 0;
          progressed = true;
        } else if (q != cudaErrorNotReady) {
          rc = SYMBA_E_CUDA;
          break;
        }
      }
      if (!busy[i] && left[i] > 0) {
        symba_pool *P = ctxs[i]->pool;
        const int r = pool_step(P, 1);
        if (r != SYMBA_OK) { rc = r; break; }
        if (cudaEventRecord(ev[i], P->stream) != cudaSuccess) { rc = SYMBA_E_CUDA; break; }
        busy[i] = 1;
        --left[i];
        progressed = true;
      }
      pending = pending || busy[i] || left[i] > 0;
    }
    if (!progressed) std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
  for (int i = 0; i < n; ++i)
    if (ev[i]) cudaEventDestroy(ev[i]);
  if (rc != SYMBA_OK) return rc;
  int worst = SYMBA_OK;
  for (int i = 0; i < n; ++i) {
    const int s = slot_status(ctxs[i]->pool, ctxs[i]->slot);
    if (s < 0 && (worst >= 0 || s < worst)) worst = s;
    else if (s > 0 && worst == SYMBA_OK) worst = s;
  }
  return worst;
}

int symba_energy(symba_ctx *c, double *E, double L[3]) {
  if (!c) return SYMBA_E_INVAL;
  return energy(c->pool, c->slot, E, L);
}

int symba_enc_groups(symba_ctx *c, int *pairs, int *group_of_pair, int cap, int *n_pairs, int *n_groups) {
  if (!c) return SYMBA_E_INVAL;
  return enc_groups(c->pool, c->slot, pairs, group_of_pair, cap, n_pairs, n_groups);
}

int symba_get_state(symba_ctx *c, double *x, double *v, double *m, double *radius, int *alive) {
  if (!c) return SYMBA_E_INVAL;
  return get_state(c->pool, c->slot, x, v, m, radius, alive);
}

int symba_get_rhill(symba_ctx *c, double *rhill) {
  if (!c) return SYMBA_E_INVAL;
  return get_rhill(c->pool, c->slot, rhill);
}

int symba_pool_get_rhill(symba_pool *pool, int slot, double *rhill) { return get_rhill(pool, slot, rhill); }

int symba_pool_set_state(symba_pool *pool, int slot, const double *x, const double *v) {
  return set_state(pool, slot, x, v);
}

int symba_pool_enc_groups(symba_pool *pool, int slot, int *pairs, int *group_of_pair, int cap, int *n_pairs,
                          int *n_groups) {
  return enc_groups(pool, slot, pairs, group_of_pair, cap, n_pairs, n_groups);
}

int symba_set_state(symba_ctx *c, const double *x, const double *v) {
  if (!c) return SYMBA_E_INVAL;
  return set_state(c->pool, c->slot, x, v);
}

int symba_get_stats(symba_ctx *c, symba_stats *s) {
  if (!c) return SYMBA_E_INVAL;
  return get_stats(c->pool, c->slot, s);
}

int symba_profile_step(symba_ctx *c, int nsteps, double *phase_ms) {
  if (!c) return SYMBA_E_INVAL;
  const int rc = pool_profile(c->pool, nsteps, phase_ms);
  if (rc != SYMBA_OK) return rc;
  return slot_status(c->pool, c->slot);
}

void symba_free(symba_ctx *c) {
  if (!c) return;
  symba_pool_free(c->pool);
  delete c;
}

}  // extern "C"
