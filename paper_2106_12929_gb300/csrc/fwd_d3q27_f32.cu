// D3Q27 kernels with float population storage (every collision, force on/off, layout).
#include "lb_kernels.cuh"

namespace lb {
cudaError_t run_op_d3q27_f32(const OpArgs& a) { return run_op_typed<D3Q27, float>(a); }
}  // namespace lb
