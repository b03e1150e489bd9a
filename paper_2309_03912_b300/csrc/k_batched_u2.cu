// k_batched_u2.cu -- the batched kernel at two 16-byte vectors per lane (the
// narrower, lower-register form the plan's autotuner can pick); the host side
// and the four-vector form are in k_batched.cu.
#include "batched_kernel.cuh"

namespace tr {

BatchedKernel batched_kernel_u2(tr_dtype xt, int threads) { return batched_kernel<2>(xt, threads); }

}  // namespace tr
