// Where a caller's array lives.  Every entry point takes host or device pointers; a device
// pointer is used in place only when it belongs to the current device (or is managed memory,
// which any device may touch).  A pointer into another GPU's memory is rejected: the kernels run
// on the current device, and without peer access dereferencing it is an illegal-address fault.
#pragma once
#include <cuda_runtime_api.h>

enum PtrClass { PTR_FOREIGN = -1, PTR_HOST = 0, PTR_DEVICE = 1 };

// The decision from the pointer's attributes and the current device (pure, testable on a host
// without a GPU).  Unregistered and page-locked host memory are host memory.
inline int classify_pointer(cudaMemoryType type, int owner_device, int current_device) {
  if (type == cudaMemoryTypeManaged) return PTR_DEVICE;
  if (type == cudaMemoryTypeDevice) return owner_device == current_device ? PTR_DEVICE : PTR_FOREIGN;
  return PTR_HOST;
}

// The class of p on the current device; NULL and pointers the runtime does not know are host.
inline int pointer_class(const void *p) {
  if (!p) return PTR_HOST;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return PTR_HOST;
  }
  int cur = 0;
  if (cudaGetDevice(&cur) != cudaSuccess) return PTR_FOREIGN;
  return classify_pointer(a.type, a.device, cur);
}
