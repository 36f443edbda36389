// Spectral flow control of Sec. 3.2 on D2Q9: host-side declarations shared by lb_api.cu
// and lb_spectral.cu.
#pragma once

#include "lb_ops.cuh"

namespace lb {

struct SpectralArgs {
    OpArgs a;                        // state to read (src, mode, storage, geometry), stream
    int n = 0, logn = 0;             // grid edge: nx = ny = n = 2^logn
    void* spec = nullptr;            // [n][n] complex values of the arithmetic type
    const void* tw = nullptr;        // [n/2] twiddle factors exp(-i 2 pi k / n), arithmetic type
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

// Largest grid edge (shared-memory FFT of one line per block).
constexpr int kSpecMaxN = 4096;

// Spectrum sigma of the state a.src; with sigma0 also the cost R and dR/dsigma; with du
// also the velocity shift du = -kappa grad_u R. Adds the number of launches to *launches.
cudaError_t spectral_shift(const SpectralArgs& s, int* launches);
// The twiddle table of the n-point DFT into tw (n/2 complex values of the storage's arithmetic
// type), once per context.
cudaError_t spectral_twiddles(void* tw, int n, int storage, cudaStream_t st);
// One controlled step from the state s.a.src into s.a.dst (s.a's mode, omega and status):
// spectrum, cost and dR/dsigma as above, then BGK at u + du with du kept on chip (s.du unused).
cudaError_t spectral_step(const SpectralArgs& s, int* launches);

}  // namespace lb
