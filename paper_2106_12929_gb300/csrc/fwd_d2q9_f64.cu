// D2Q9 kernels with double population storage (every collision, force on/off, layout).
#include "lb_kernels.cuh"

namespace lb {
cudaError_t run_op_d2q9_f64(const OpArgs& a) { return run_op_typed<D2Q9, double>(a); }
}  // namespace lb
