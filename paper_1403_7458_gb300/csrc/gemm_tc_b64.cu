// gemm_tc_b64.cu -- the tcgen05 leaf-product kernel (tc_kernel.cuh)
// instantiated for leaf 64 (its own translation unit so that the leaf sizes
// compile in parallel).
#include "tc_kernel.cuh"

int tc_launch_b64(const tc::TcArgs &a, int S, int E, cudaStream_t s) { return tc::launch_leaf<64>(a, S, E, s); }
