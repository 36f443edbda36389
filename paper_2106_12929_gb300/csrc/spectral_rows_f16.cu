// Row kernels of the spectral flow control (Sec. 3.2) for __half population storage, every grid
// edge 4 ... 4096 (one translation unit per storage type so that the sizes compile in parallel).
#include "lb_spectral_fft.cuh"

namespace lb {
cudaError_t spectral_rows_f16(const SpectralArgs& s, bool step) { return sc::rows_typed<__half>(s, step); }
}  // namespace lb
