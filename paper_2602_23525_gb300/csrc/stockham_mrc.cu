// stockham_mrc.cu -- the mixed-radix Stockham pass kernel (gb_mr_kernel.cuh)
// with compile-time radix schedules for the lengths that batched workloads
// use most: the planner's own schedules for 1000 = 8 5 5 5, 2187 = 9 9 9 3,
// 3125 = 5^5 (this unit), 3600 = 16 9 5 5, 3840 = 16 16 3 5 and 7168 =
// 16 16 4 7 (stockham_mrc2.cu, compiled in parallel).  A plan whose length
// and schedule match one of them launches it instead of the run-time
// schedule; the tiles, copies and stores are the same kernel's.
#include "gb_mr_static.cuh"

int gb_mr_dispatch_static_a(const GbMR& k, cudaStream_t st, cudaError_t* e) {
  return try_static<MRS<8, 5, 5, 5>>(k, st, e) || try_static<MRS<9, 9, 9, 3>>(k, st, e) ||
         try_static<MRS<5, 5, 5, 5, 5>>(k, st, e);
}

int gb_mr_dispatch_static(const GbMR& k, cudaStream_t st, cudaError_t* e) {
  return gb_mr_dispatch_static_a(k, st, e) || gb_mr_dispatch_static_b(k, st, e);
}
