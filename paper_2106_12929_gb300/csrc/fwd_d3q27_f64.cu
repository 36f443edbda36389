// D3Q27 kernels with double population storage (every collision, force on/off, layout).
#include "lb_kernels.cuh"

namespace lb {
cudaError_t run_op_d3q27_f64(const OpArgs& a) { return run_op_typed<D3Q27, double>(a); }
}  // namespace lb
