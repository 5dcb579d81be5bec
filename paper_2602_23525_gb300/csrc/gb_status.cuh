// gb_status.cuh -- how a kernel reports a device-side error to its plan.
//
// A plan's status word lives in page-locked host memory mapped into the
// device's address space, so the host can read it at any time without
// synchronising the device.  Kernels only ever store one error code there
// (all writers store the same value), with a plain volatile store made
// visible system-wide; the host clears it when it collects the error.
#pragma once
#include <cuda_runtime.h>

__device__ __forceinline__ void gb_set_status(int* status, int code) {
  if (!status) return;
  *reinterpret_cast<volatile int*>(status) = code;
  __threadfence_system();
}
