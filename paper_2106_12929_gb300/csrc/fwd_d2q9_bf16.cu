// D2Q9 kernels with __nv_bfloat16 population storage (every collision, force on/off, layout).
#include "lb_kernels.cuh"

namespace lb {
cudaError_t run_op_d2q9_bf16(const OpArgs& a) { return run_op_typed<D2Q9, __nv_bfloat16>(a); }
}  // namespace lb
