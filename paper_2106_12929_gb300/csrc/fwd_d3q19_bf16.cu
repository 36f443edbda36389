// D3Q19 kernels with __nv_bfloat16 population storage (every collision, force on/off, layout).
#include "lb_kernels.cuh"

namespace lb {
cudaError_t run_op_d3q19_bf16(const OpArgs& a) { return run_op_typed<D3Q19, __nv_bfloat16>(a); }
}  // namespace lb
