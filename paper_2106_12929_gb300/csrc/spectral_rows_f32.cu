// Row kernels of the spectral flow control (Sec. 3.2) for float population storage, every grid
// edge 4 ... 4096 (one translation unit per storage type so that the sizes compile in parallel).
#include "lb_spectral_fft.cuh"

namespace lb {
cudaError_t spectral_rows_f32(const SpectralArgs& s, bool step) { return sc::rows_typed<float>(s, step); }
}  // namespace lb
