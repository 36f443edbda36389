// Row kernels of the spectral flow control (Sec. 3.2) for __nv_bfloat16 population storage, every grid
// edge 4 ... 4096 (one translation unit per storage type so that the sizes compile in parallel).
#include "lb_spectral_fft.cuh"

namespace lb {
cudaError_t spectral_rows_bf16(const SpectralArgs& s, bool step) { return sc::rows_typed<__nv_bfloat16>(s, step); }
}  // namespace lb
