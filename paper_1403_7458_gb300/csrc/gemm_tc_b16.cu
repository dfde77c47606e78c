// gemm_tc_b16.cu -- the tcgen05 leaf-product kernel (tc_kernel.cuh)
// instantiated for leaf 16 (its own translation unit so that the leaf sizes
// compile in parallel).
#include "tc_kernel.cuh"

int tc_launch_b16(const tc::TcArgs &a, int S, int E, cudaStream_t s) { return tc::launch_leaf<16>(a, S, E, s); }
