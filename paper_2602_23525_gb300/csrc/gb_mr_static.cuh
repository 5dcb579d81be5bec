// gb_mr_static.cuh -- launch of the mixed-radix pass kernel with a
// compile-time radix schedule (MRS in gb_mr_kernel.cuh), shared by the
// translation units that instantiate the schedules.
#pragma once
#include "gb_mr_kernel.cuh"

int gb_mr_dispatch_static_a(const GbMR& k, cudaStream_t st, cudaError_t* e);
int gb_mr_dispatch_static_b(const GbMR& k, cudaStream_t st, cudaError_t* e);

namespace {

// launches k with schedule SCH when its length and schedule are SCH's
template <class SCH>
bool try_static(const GbMR& k, cudaStream_t st, cudaError_t* e) {
  if (!SCH::matches(k)) return false;
  if (k.T * k.tpt <= 256) *e = dispatch<256, SCH>(k, st);
  else if (k.T * k.tpt <= 512) *e = dispatch<512, SCH>(k, st);
  else *e = cudaErrorInvalidValue;
  return true;
}

}  // namespace
