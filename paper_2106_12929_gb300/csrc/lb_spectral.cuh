// Spectral flow control of Sec. 3.2 on D2Q9: host-side declarations shared by lb_api.cu,
// lb_spectral.cu and the row-kernel units spectral_rows_<type>.cu.
#pragma once

#include "lb_ops.cuh"

namespace lb {

struct SpectralArgs {
    OpArgs a;                        // state to read (src, mode, storage, geometry), stream
    int n = 0, logn = 0;             // grid edge: nx = ny = n = 2^logn
    void* spec = nullptr;            // [n][n] complex values of the arithmetic type
    const void* tw = nullptr;        // level twiddle factors (arithmetic type), spectral_twiddle_count(n)
    const void* shell = nullptr;     // [n][n] int16: round(|k|) of every mode [ky][kx]
    const void* first = nullptr;     // [n/2 + 1][n/2 + 1] int16: first |ky| of shell s in column |kx|
    double* partials = nullptr;      // [n/2][column blocks] shell sums of each block of kx columns
    double* sigma = nullptr;         // [n/2] spectrum of the state
    double* grad = nullptr;          // [n/2] dR/dsigma
    double* r2 = nullptr;            // [n/2] terms of R
    double* cost = nullptr;          // [1] R
    const double* sigma0 = nullptr;  // [n/2] target spectrum (null: spectrum only)
    const double* l0 = nullptr;      // [n/2] ln max(sigma0, cutoff), set with sigma0
    double cutoff = 2e-5, kappa = 5e-5;
    void* du = nullptr;              // [2][plane] arithmetic type: -kappa grad_u R (null: no shift)
};

// Largest grid edge (one grid line per shared-memory buffer of a block).
constexpr int kSpecMaxN = 4096;

// Spectrum sigma of the state a.src; with sigma0 also the cost R and dR/dsigma; with du
// also the velocity shift du = -kappa grad_u R. Adds the number of launches to *launches.
cudaError_t spectral_shift(const SpectralArgs& s, int* launches);
// One controlled step from the state s.a.src into s.a.dst (s.a's mode, omega and status):
// spectrum, cost and dR/dsigma as above, then BGK at u + du with du kept on chip (s.du unused).
cudaError_t spectral_step(const SpectralArgs& s, int* launches);
// Number of complex twiddle factors of the n-point line transforms.
size_t spectral_twiddle_count(int n);
// The per-context tables of grid edge n: twiddles (storage's arithmetic type), shell of every
// mode and first |ky| of every shell per column (int16 each). Adds its launches to *launches.
cudaError_t spectral_tables(void* tw, void* shell, void* first, int n, int storage, cudaStream_t st, int* launches);
// The row kernels of one storage type: moments and forward DFT along x (step = false), or the
// inverse DFT along x fused with the shifted step.
cudaError_t spectral_rows_f64(const SpectralArgs& s, bool step);
cudaError_t spectral_rows_f32(const SpectralArgs& s, bool step);
cudaError_t spectral_rows_f16(const SpectralArgs& s, bool step);
cudaError_t spectral_rows_bf16(const SpectralArgs& s, bool step);

}  // namespace lb
