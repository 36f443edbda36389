// Interface between the C-ABI host code and the per-stencil kernel translation
// units. Host-only declarations; no kernels here.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

#include "lb_device.cuh"

namespace lb {

enum Op {
    OP_UPDATE = 0,          // one fused stream + collide step (src -> dst, or in place for AA)
    OP_INIT_EQ = 1,         // state <- f^eq(rho = in0, u = in1)
    OP_SET = 2,             // state <- f (in0, natural layout)
    OP_GET = 3,             // out0 <- f (natural layout) of the state
    OP_MOMENTS = 4,         // out0 <- rho, out1 <- u of the state
    OP_REDUCE_PARTIAL = 5,  // partials[block][6] of the global sums
    OP_ADJ_SEED = 6,        // out0 <- lambda from (in0 = dL/drho or null, in1 = dL/du); gF += direct part
    OP_ADJ_STEP = 7,        // lam_out <- J^T S^T lam_in at state src; gF += force part
    OP_LOSS_ENERGY = 8,     // per-node energy loss seed (in0 = e*), partials[block] = sum of squares
    OP_LINKS = 9,           // out0 <- bounce-back links of every node from the solid mask in0 (uint8)
};

// storage codes match lb_storage
enum StorageCode { S_F64 = 0, S_F32 = 1, S_F16 = 2, S_BF16 = 3 };

struct OpArgs {
    int op = OP_UPDATE;
    int storage = S_F32;
    int coll = 0;
    int force = 0;
    int mode = AB;
    const void* src = nullptr;  // population buffer holding the state
    void* dst = nullptr;        // population buffer written (UPDATE: next state; SET/INIT: state)
    const void* F = nullptr;    // force [D][plane], arithmetic type
    const void* in0 = nullptr;
    const void* in1 = nullptr;
    void* out0 = nullptr;
    void* out1 = nullptr;
    int io_f64 = 1;             // caller arrays are FP64 (1) or FP32 (0)
    const void* lam_in = nullptr;   // adjoint: lambda^{n+1} [Q][plane], arithmetic type
    void* lam_out = nullptr;        // adjoint: lambda^n
    void* gF = nullptr;             // adjoint: force gradient accumulator [D][plane], arithmetic type
    void* gth = nullptr;            // learned adjoint: per-block network-gradient partials
    const void* tc_table = nullptr; // learned collision on tensor cores: packed weight table (device)
    const void* x3_table = nullptr; // learned collision, FP32 arithmetic: split BF16 weight table (device)
    Geom g{};
    double omega = 1.0;
    double rx[3] = {0.0, 0.0, 0.0};  // further constants of the collision (lb_collide.cuh, Relax)
    int npt = 0;                     // stream-collide nodes per thread: 0 = from the grid, 1, 2, 4
    int sms = 0;                     // multiprocessors of the device
    unsigned* status = nullptr;
    double* partials = nullptr;
    cudaStream_t stream = nullptr;
};

// grid of the node kernels: blocks of up to 128 threads along x, one block row per (y, z)
inline dim3 node_block(const Geom& g)
{
    int bx = g.nx >= 128 ? 128 : ((g.nx + 31) / 32) * 32;
    return dim3(bx, 1, 1);
}
inline dim3 node_grid(const Geom& g)
{
    dim3 b = node_block(g);
    return dim3((g.nx + b.x - 1) / b.x, g.ny, g.nz);
}
inline int64_t node_grid_blocks(const Geom& g)
{
    dim3 gr = node_grid(g);
    return (int64_t)gr.x * gr.y * gr.z;
}

cudaError_t run_op_d2q9_f64(const OpArgs& a);
cudaError_t run_op_d2q9_f32(const OpArgs& a);
cudaError_t run_op_d2q9_f16(const OpArgs& a);
cudaError_t run_op_d2q9_bf16(const OpArgs& a);
cudaError_t run_op_d3q19_f64(const OpArgs& a);
cudaError_t run_op_d3q19_f32(const OpArgs& a);
cudaError_t run_op_d3q19_f16(const OpArgs& a);
cudaError_t run_op_d3q19_bf16(const OpArgs& a);
cudaError_t run_op_d3q27_f64(const OpArgs& a);
cudaError_t run_op_d3q27_f32(const OpArgs& a);
cudaError_t run_op_d3q27_f16(const OpArgs& a);
cudaError_t run_op_d3q27_bf16(const OpArgs& a);

// one entry per (stencil, storage); defined in fwd_<stencil>_<storage>.cu
inline cudaError_t run_op(int stencil, const OpArgs& a)
{
    using Fn = cudaError_t (*)(const OpArgs&);
    static const Fn table[3][4] = {
        {run_op_d2q9_f64, run_op_d2q9_f32, run_op_d2q9_f16, run_op_d2q9_bf16},
        {run_op_d3q19_f64, run_op_d3q19_f32, run_op_d3q19_f16, run_op_d3q19_bf16},
        {run_op_d3q27_f64, run_op_d3q27_f32, run_op_d3q27_f16, run_op_d3q27_bf16}};
    if (stencil < 0 || stencil > 2 || a.storage < 0 || a.storage > 3) return cudaErrorInvalidValue;
    return table[stencil][a.storage](a);
}

// message returned by lb_last_error() on the calling thread (lb_api.cu)
void set_last_error(const char* msg);

// stencil-independent helpers (lb_aux.cu)
cudaError_t reduce_final(const double* partials, int64_t nblocks, int width, double* out, cudaStream_t s);
// dst <- src, bytes a multiple of 16 with 16-byte aligned device pointers (bandwidth reference)
cudaError_t stream_copy(const void* src, void* dst, int64_t bytes, int sms, cudaStream_t s);
cudaError_t convert_copy(const void* src, int src_f64, void* dst, int dst_f64, int64_t n, int64_t src_stride,
                         int64_t dst_stride, int rows, int accumulate, cudaStream_t s);
cudaError_t coarsen2(const double* rho_f, const double* u_f, int nxf, int nyf, int nzf, int d, double* rho_c,
                     double* u_c, cudaStream_t s);
cudaError_t vorticity2d(const double* u, int nx, int ny, void* w, int w_f64, cudaStream_t s);
cudaError_t adam_update(float* theta, float* m, float* v, const float* grad, int64_t n, float lr, float b1,
                        float b2, float eps, float c1, float c2, cudaStream_t s);

}  // namespace lb
