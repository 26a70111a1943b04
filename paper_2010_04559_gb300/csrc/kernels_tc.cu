// placeholder, replaced by the tcgen05 kernel
#include "kernels.cuh"
namespace amgt {
bool tc_available() { return false; }
int launch_tc_gemm(int, int, int, const __nv_bfloat16*, const __nv_bfloat16*, float*,
                   const GemmEpi&, int*, cudaStream_t) { return -1; }
}  // namespace amgt
