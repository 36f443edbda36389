// Learned moment-space collision on D2Q9 (Eq. 5, Sec. 3.1) and the Eq. 6 loss:
// host-side declarations shared by lb_api.cu and lb_learned.cu.
#pragma once

#include "lb_ops.cuh"

namespace lb {

constexpr int kNetIn = 6, kNetHidden = 24;
constexpr int kNetTheta = kNetHidden * kNetIn + kNetHidden + kNetHidden * kNetHidden + kNetHidden + kNetHidden + 1;
constexpr int kNetValues = kNetTheta + 2 * kNetIn;  // + input shift and scale
static_assert(kNetTheta == 793, "6-24-24-1 network has 793 parameters");
// the network shape Sec. 3.1 describes: one hidden layer, three outputs (one relaxation
// time per higher moment)
constexpr int kNet3Hidden = 53;
constexpr int kNet3Theta = kNet3Hidden * kNetIn + kNet3Hidden + 3 * kNet3Hidden + 3;
constexpr int kNet3Values = kNet3Theta + 2 * kNetIn;
static_assert(kNet3Theta == 533, "6-53-3 network has 533 parameters");

// forward step / adjoint step of the learned collision (a.op = OP_UPDATE or OP_ADJ_STEP);
// net = kNetValues host doubles; a.gth = per-block parameter-gradient partials (adjoint).
// FP64 storage runs the scalar FP64 kernels, the other storage types the tensor-core
// kernels of the FP32 arithmetic (run_learned_x3); tc = 1: forward step with the network in
// half precision instead (the learned_tc inference option, run_learned_tc)
cudaError_t run_learned_d2q9(const OpArgs& a, const double* net, bool tc = false);
// the same for the one-hidden-layer network with three outputs (net = kNet3Values doubles)
cudaError_t run_learned3_d2q9(const OpArgs& a, const double* net, bool tc = false);
// The learned_tc inference option (lb_learned_tc.cu): weights packed once per lb_set_mlp
// into a device table (bytes needed, host-side packing into `out`), and the forward step
// (a.tc_table; needs 9 x plane < 2^31).
size_t learned_tc_table_bytes();
void learned_tc_pack(const double* net, void* out);
size_t learned3_tc_table_bytes();
void learned3_tc_pack(const double* net, void* out);
cudaError_t run_learned_tc(const OpArgs& a, bool three);
// out[6][N] <- the six network inputs (moment invariants) of every node of the state a.src
cudaError_t learned_inputs_d2q9(const OpArgs& a);
// FP32 arithmetic (FP32 / FP16 / BF16 storage): the networks on the tensor cores with
// split BF16 operands (lb_learned_x3.cu). Weight table bytes and host packing (once per
// lb_set_mlp), the forward / adjoint step (a.x3_table), and the rows of its gradient partials.
size_t learned_x3_table_bytes(bool three);
void learned_x3_pack(const double* net, bool three, void* out);
cudaError_t run_learned_x3(const OpArgs& a, bool three);
int64_t learned_x3_partial_count(const Geom& g, int storage, int sms, bool three);
// rows of the gradient partials of the learned adjoint launch (blocks of the launch)
int64_t learned_adj_partial_count(const Geom& g, int storage, int sms, bool three);
// out[ntheta] (+)= sum over blocks of partials[block][ntheta] (two deterministic passes
// through `chunk`, learned_theta_chunk_doubles() doubles of scratch; ntheta <= kNetTheta)
int64_t learned_theta_chunk_doubles();
cudaError_t learned_reduce_theta(const void* partials, int64_t nblk, int ntheta, int part_f64, double* chunk,
                                 void* out, int out_f64, cudaStream_t s);

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
