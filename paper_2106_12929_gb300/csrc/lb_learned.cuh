// Learned moment-space collision on D2Q9 (Eq. 5, Sec. 3.1) and the Eq. 6 loss:
// host-side declarations shared by lb_api.cu and lb_learned.cu.
#pragma once

#include "lb_ops.cuh"

namespace lb {

constexpr int kNetIn = 6, kNetHidden = 24;
constexpr int kNetTheta = kNetHidden * kNetIn + kNetHidden + kNetHidden * kNetHidden + kNetHidden + kNetHidden + 1;
constexpr int kNetValues = kNetTheta + 2 * kNetIn;  // + input shift and scale
static_assert(kNetTheta == 793, "6-24-24-1 network has 793 parameters");

// forward step / adjoint step of the learned collision (a.op = OP_UPDATE or OP_ADJ_STEP);
// net = kNetValues host doubles; a.gth = per-block parameter-gradient partials (adjoint)
// tc = 1: forward step with the network's hidden layers on the tensor cores (BF16 x BF16 -> FP32)
cudaError_t run_learned_d2q9(const OpArgs& a, const double* net, bool tc = false);
// Network weights for the tensor-core path, packed once per lb_set_mlp into a device table:
// bytes needed, and the host-side packing into `out` (learned_tc_table_bytes() bytes).
size_t learned_tc_table_bytes();
void learned_tc_pack(const double* net, void* out);
// out[6][N] <- the six network inputs (moment invariants) of every node of the state a.src
cudaError_t learned_inputs_d2q9(const OpArgs& a);
// number of blocks of the learned adjoint launch (rows of the gradient partials)
int64_t learned_adj_partial_count(const Geom& g);
// out[793] (+)= sum over blocks of partials[block][793] (two deterministic passes through
// `chunk`, learned_theta_chunk_doubles() doubles of scratch)
int64_t learned_theta_chunk_doubles();
cudaError_t learned_reduce_theta(const void* partials, int64_t nblk, int part_f64, double* chunk, void* out,
                                 int out_f64, cudaStream_t s);

struct LossEq6Args {
    OpArgs a;                    // state, geometry, stream
    const void* uref = nullptr;  // [2][N] caller dtype
    const void* wref = nullptr;  // [N]
    double Eref = 0.0;
    void* lam = nullptr;         // [9][N] caller dtype, may be null
    int io_f64 = 1;
    double* partials = nullptr;  // >= 3 * blocks + 8 doubles
    double* result = nullptr;    // device double: the loss
    void* scratch = nullptr;     // [3][plane] arithmetic type
    int64_t N = 0;
};
cudaError_t loss_eq6_d2q9(const LossEq6Args& e, int* launches);

}  // namespace lb
