// Energy and angular momentum without any device allocation (symba_energy_static).
//
// Some callers cannot allocate device memory: a host loop with a hard per-iteration latency
// budget cannot afford cudaMalloc/cudaFree (they may synchronise the whole device), and a process
// whose device memory belongs to another allocator (a framework's caching allocator, or a fixed
// memory budget) must not take any.  This entry point computes the same sums as symba_energy
// from caller-owned device arrays; the exact-sum accumulator it needs lives in the file-scope
// array below, which every GPU that loads the library holds until the process exits.
//
// The accumulator slots are 64-bit carry-save digits that each absorb at most 2^31 - 1
// additions of 32-bit chunks, so a call may sum at most 2^31 - 1 terms into one accumulator: the
// energy takes n (n - 1)/2 + 2n + 1 of them for n bodies, hence the limit
// SYMBA_ENERGY_STATIC_MAX_N = 65,534 (checked below at compile time).
#include <algorithm>

#include "internal.cuh"
#include "ptr_class.h"

constexpr long long energy_terms(long long n) { return n * (n - 1) / 2 + 2 * n + 1; }
static_assert(energy_terms(SYMBA_ENERGY_STATIC_MAX_N) <= 2147483647LL,
              "the energy accumulator of the largest accepted n must take at most 2^31 - 1 terms");
static_assert(energy_terms(SYMBA_ENERGY_STATIC_MAX_N + 1) > 2147483647LL,
              "SYMBA_ENERGY_STATIC_MAX_N is the largest n the accumulator allows");

// 7 accumulators (E, Lx, Ly, Lz, Px, Py, Pz) of SA_NDIG + 1 slots: 3,864 bytes
#define STATIC_ACCS 7
static __device__ __align__(256) unsigned long long g_static_energy_scratch[STATIC_ACCS * (SA_NDIG + 1)];

namespace {

// Device address of the scratch array on the current device.  In host code the array's name is
// a host-side stand-in, not a device address, so the address is asked of the runtime (with that
// device current) at every call: the lookup allocates nothing, and a module reloaded after a
// device reset gets its new address instead of a stale cached one.  The first lookup on a device
// may load the module, which is why the first call there should precede any stream capture.
int scratch_address(unsigned long long **out) {
  void *ptr = nullptr;
  if (cudaGetSymbolAddress(&ptr, g_static_energy_scratch) != cudaSuccess) return SYMBA_E_CUDA;
  *out = (unsigned long long *)ptr;
  return SYMBA_OK;
}

// a device array of the current device (or managed memory); host arrays and other GPUs' arrays
// are refused
bool on_device(const void *p) { return pointer_class(p) == PTR_DEVICE; }

}  // namespace

__global__ void k_static_clear(unsigned long long *acc) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < STATIC_ACCS * (SA_NDIG + 1); k += gridDim.x * blockDim.x)
    acc[k] = 0ull;
}

// per body: kinetic and solar terms, L, and the momentum sum P (same operation order as the
// pool path: (0.5 m) v^2, -(G m0) m / r, m (x_c1 v_c2 - x_c2 v_c1), m v_c)
__global__ void __launch_bounds__(256) k_static_bodies(int n, const double *x, const double *v,
                                                       const double *m, double G, double m0,
                                                       unsigned long long *acc) {
  __shared__ unsigned long long s[STATIC_ACCS][SA_NDIG + 1];
  for (int k = threadIdx.x; k < STATIC_ACCS * (SA_NDIG + 1); k += blockDim.x) (&s[0][0])[k] = 0ull;
  __syncthreads();
  const double Gm0 = __dmul_rn(G, m0);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double mi = m[i];
    const double px = x[3 * i], py = x[3 * i + 1], pz = x[3 * i + 2];
    const double ux = v[3 * i], uy = v[3 * i + 1], uz = v[3 * i + 2];
    const double v2 = __dadd_rn(__dadd_rn(__dmul_rn(ux, ux), __dmul_rn(uy, uy)), __dmul_rn(uz, uz));
    sa_add(s[0], __dmul_rn(__dmul_rn(0.5, mi), v2));
    const double r = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(px, px), __dmul_rn(py, py)), __dmul_rn(pz, pz)));
    sa_add(s[0], -__ddiv_rn(__dmul_rn(Gm0, mi), r));
    sa_add(s[1], __dmul_rn(mi, __dsub_rn(__dmul_rn(py, uz), __dmul_rn(pz, uy))));
    sa_add(s[2], __dmul_rn(mi, __dsub_rn(__dmul_rn(pz, ux), __dmul_rn(px, uz))));
    sa_add(s[3], __dmul_rn(mi, __dsub_rn(__dmul_rn(px, uy), __dmul_rn(py, ux))));
    if (mi != 0.0) {
      sa_add(s[4], __dmul_rn(mi, ux));
      sa_add(s[5], __dmul_rn(mi, uy));
      sa_add(s[6], __dmul_rn(mi, uz));
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < STATIC_ACCS * (SA_NDIG + 1); k += blockDim.x) {
    const unsigned long long val = (&s[0][0])[k];
    if (val) atomicAdd(&acc[k], val);
  }
}

// pair potential over the trapezoid i < n_massive, j > i, one warp per 32 x 32 block
__global__ void __launch_bounds__(256) k_static_pairs(int n, int nm, const double *x, const double *m,
                                                      double G, unsigned long long *acc) {
  __shared__ unsigned long long s[SA_NDIG + 1];
  for (int k = threadIdx.x; k < SA_NDIG + 1; k += blockDim.x) s[k] = 0ull;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int nb = (n + 31) / 32, nbm = (nm + 31) / 32;
  const long long nt = (long long)nbm * nb;
  const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long t = warp; t < nt; t += nwarps) {
    const int I = (int)(t / nb), J = (int)(t % nb);
    if (J < I) continue;
    const int i = I * 32 + lane;
    if (i >= nm || i >= n) continue;
    const double xi = x[3 * i], yi = x[3 * i + 1], zi = x[3 * i + 2];
    const double Gmi = __dmul_rn(G, m[i]);
    for (int k = 0; k < 32; ++k) {
      const int j = J * 32 + k;
      if (j <= i || j >= n) continue;
      const double dx = __dsub_rn(x[3 * j], xi), dy = __dsub_rn(x[3 * j + 1], yi), dz = __dsub_rn(x[3 * j + 2], zi);
      const double r = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)));
      sa_add(s, -__ddiv_rn(__dmul_rn(Gmi, m[j]), r));
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < SA_NDIG + 1; k += blockDim.x) {
    const unsigned long long val = s[k];
    if (val) atomicAdd(&acc[k], val);
  }
}

// |P|^2 / (2 m0) with P rounded from its exact sums, then E, L rounded into out[0..3]
__global__ void k_static_finish(double m0, unsigned long long *acc, double *out) {
  if (threadIdx.x != 0) return;
  const double Px = sa_round(acc + 4 * (SA_NDIG + 1));
  const double Py = sa_round(acc + 5 * (SA_NDIG + 1));
  const double Pz = sa_round(acc + 6 * (SA_NDIG + 1));
  const double P2 = __dadd_rn(__dadd_rn(__dmul_rn(Px, Px), __dmul_rn(Py, Py)), __dmul_rn(Pz, Pz));
  sa_add(acc, __ddiv_rn(P2, __dmul_rn(2.0, m0)));
  for (int k = 0; k < 4; ++k) out[k] = sa_round(acc + k * (SA_NDIG + 1));
}

extern "C" int symba_energy_static(int n, int n_massive, const double *x, const double *v,
                                   const double *m, double G, double m0, double *out,
                                   void *cuda_stream) {
  if (n < 1 || n_massive < 0 || n_massive > n || !x || !v || !m || !out || !(m0 > 0.0))
    return SYMBA_E_INVAL;
  if (n > SYMBA_ENERGY_STATIC_MAX_N) return SYMBA_E_INVAL;
  if (!on_device(x) || !on_device(v) || !on_device(m) || !on_device(out)) return SYMBA_E_INVAL;
  unsigned long long *acc = nullptr;
  const int st = scratch_address(&acc);
  if (st != SYMBA_OK) return st;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  int dev = 0, sms = 1;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return SYMBA_E_CUDA;
  k_static_clear<<<2, 256, 0, s>>>(acc);
  const int bb = (int)std::min<long long>((n + 255) / 256, 64);
  k_static_bodies<<<bb, 256, 0, s>>>(n, x, v, m, G, m0, acc);
  if (n_massive > 0) k_static_pairs<<<sms * 4, 256, 0, s>>>(n, n_massive, x, m, G, acc);
  k_static_finish<<<1, 32, 0, s>>>(m0, acc, out);
  return cudaGetLastError() == cudaSuccess ? SYMBA_OK : SYMBA_E_CUDA;
}
