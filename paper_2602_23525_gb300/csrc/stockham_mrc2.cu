// stockham_mrc2.cu -- compile-time radix schedules of the mixed-radix pass
// kernel for 3600 = 16 9 5 5, 3840 = 16 16 3 5 and 7168 = 16 16 4 7 (the
// rest, and the dispatch, are in stockham_mrc.cu).
#include "gb_mr_static.cuh"

int gb_mr_dispatch_static_b(const GbMR& k, cudaStream_t st, cudaError_t* e) {
  return try_static<MRS<16, 9, 5, 5>>(k, st, e) || try_static<MRS<16, 16, 3, 5>>(k, st, e) ||
         try_static<MRS<16, 16, 4, 7>>(k, st, e);
}
