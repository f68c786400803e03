// Device rates that bound this path's kernels, measured on the device the library runs on
// (symba_measure_rates).  Neither the pair kick nor the group recursion is a dense contraction,
// so no tensor-core peak applies: the kick is bound by the FP64 pipe, the recursion by how fast
// one warp completes dependent FP64 work.  The benchmark divides by these measured figures.
//
//   k_rate_dfma   every SM busy with independent FP64 fused multiply-adds (8 chains per thread,
//                 8 warps per SM): the chip's FP64 rate in FLOP/s (an FMA counts 2).
//   k_rate_warp   one warp alone: cycles per FP64 FMA in one dependent chain, and per FMA when
//                 four independent chains are interleaved (equal when the limit is per warp, not
//                 the dependency).
//   k_rate_bar    two warps of one CTA handing a value back and forth through shared memory with
//                 hardware named barriers (bar.sync with a thread count of 64): cycles per round
//                 trip.  Both warps run the same fixed number of barriers, so every wait ends.
#include "internal.cuh"

#define RATE_CHAINS 8
#define RATE_ITERS 2048

__global__ void __launch_bounds__(256) k_rate_dfma(double b, double c, double *sink) {
  double a[RATE_CHAINS];
#pragma unroll
  for (int k = 0; k < RATE_CHAINS; ++k) a[k] = (double)(threadIdx.x + k) * 1e-3;
  for (int it = 0; it < RATE_ITERS; ++it) {
#pragma unroll
    for (int k = 0; k < RATE_CHAINS; ++k) a[k] = fma(a[k], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < RATE_CHAINS; ++k) s += a[k];
  if (s == 12345.678) sink[blockIdx.x] = s;   // never true: keeps the chains alive
}

__global__ void k_rate_warp(double b, double c, long long *cycles, double *sink) {
  double a0 = threadIdx.x * 1e-3, a1 = a0 + 1.0, a2 = a0 + 2.0, a3 = a0 + 3.0;
  __syncwarp();
  long long t0 = clock64();
  for (int it = 0; it < RATE_ITERS; ++it) a0 = fma(a0, b, c);
  __syncwarp();
  long long t1 = clock64();
  for (int it = 0; it < RATE_ITERS / 4; ++it) {
    a0 = fma(a0, b, c);
    a1 = fma(a1, b, c);
    a2 = fma(a2, b, c);
    a3 = fma(a3, b, c);
  }
  __syncwarp();
  long long t2 = clock64();
  if (threadIdx.x == 0) {
    cycles[0] = t1 - t0;
    cycles[1] = t2 - t1;
  }
  if (a0 + a1 + a2 + a3 == 12345.678) sink[0] = a0;
}

__global__ void k_rate_bar(long long *cycles, int rounds) {
  __shared__ volatile int box[2];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) { box[0] = 0; box[1] = 0; }
  __syncthreads();
  long long t0 = clock64();
  for (int r = 0; r < rounds; ++r) {
    if (warp == 0 && lane == 0) box[0] = box[1] + 1;
    asm volatile("bar.sync 1, 64;" ::: "memory");
    if (warp == 1 && lane == 0) box[1] = box[0] + 1;
    asm volatile("bar.sync 2, 64;" ::: "memory");
  }
  long long t1 = clock64();
  if (threadIdx.x == 0) {
    cycles[0] = t1 - t0;
    cycles[1] = box[1];
  }
}

extern "C" int symba_measure_rates(double *out) {
  if (!out) return SYMBA_E_INVAL;
  int dev = 0, sms = 1, clk_khz = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return SYMBA_E_CUDA;
  cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, dev);
  const int blocks = sms * 2, threads = 256;   // 8 warps per SM
  double *sink = nullptr;
  long long *cyc = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = SYMBA_OK;
  if (cudaMalloc(&sink, sizeof(double) * blocks) != cudaSuccess ||
      cudaMalloc(&cyc, sizeof(long long) * 4) != cudaSuccess) rc = SYMBA_E_NOMEM;
  if (rc == SYMBA_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
    rc = SYMBA_E_CUDA;
  float best_ms = 1e30f;
  if (rc == SYMBA_OK) {
    for (int rep = 0; rep < 6; ++rep) {       // first launch warms up; best of the rest
      cudaEventRecord(e0, 0);
      k_rate_dfma<<<blocks, threads>>>(0.9999999, 1e-8, sink);
      cudaEventRecord(e1, 0);
      float ms = 0.f;
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
        rc = SYMBA_E_CUDA;
        break;
      }
      if (rep > 0 && ms < best_ms) best_ms = ms;
    }
  }
  long long h[4] = {0, 0, 0, 0};
  if (rc == SYMBA_OK) {
    k_rate_warp<<<1, 32>>>(0.9999999, 1e-8, cyc, sink);
    k_rate_warp<<<1, 32>>>(0.9999999, 1e-8, cyc, sink);
    k_rate_bar<<<1, 64>>>(cyc + 2, 1024);
    if (cudaMemcpy(h, cyc, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) rc = SYMBA_E_CUDA;
  }
  if (rc == SYMBA_OK) {
    const double flops = 2.0 * RATE_CHAINS * (double)RATE_ITERS * blocks * threads;
    out[0] = flops / (best_ms * 1e-3);                         // FP64 FLOP/s, whole device
    out[1] = (double)h[0] / RATE_ITERS;                        // cycles per dependent FMA, one warp
    out[2] = (double)h[1] / RATE_ITERS;                        // cycles per FMA, 4 chains, one warp
    out[3] = (double)h[2] / 1024.0;                            // cycles per named-barrier round trip
    out[4] = (double)sms;
    out[5] = 1e3 * (double)clk_khz;                            // the device's nominal SM clock, Hz
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(sink);
  cudaFree(cyc);
  if (rc == SYMBA_OK && cudaGetLastError() != cudaSuccess) rc = SYMBA_E_CUDA;
  return rc;
}
