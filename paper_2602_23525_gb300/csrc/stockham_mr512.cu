// stockham_mr512.cu -- the 512-thread instantiations of the mixed-radix
// Stockham pass kernel (gb_mr_kernel.cuh), compiled apart from the
// 256-thread ones so the two build in parallel.
#include "gb_mr_kernel.cuh"

cudaError_t gb_mr_dispatch_512(const GbMR& k, cudaStream_t st) { return dispatch<512>(k, st); }
