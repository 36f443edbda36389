// C-ABI of liblb (declared in include/lb.h): context management, argument
// checking, host/device staging, kernel dispatch, checkpointed adjoint driver.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "lb.h"
#include "lb_ops.cuh"
#include "lb_learned.cuh"
#include "lb_spectral.cuh"

namespace {

thread_local std::string g_last_error;

lb_status fail(lb_status s, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return s;
}

int storage_bytes(int s) { return s == LB_F64 ? 8 : (s == LB_F32 ? 4 : 2); }
int real_bytes(int s) { return s == LB_F64 ? 8 : 4; }

// Make the context's device current for the lifetime of the guard.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

}  // namespace

namespace lb {
void set_last_error(const char* msg) { g_last_error = msg; }
}  // namespace lb

struct lb_ctx {
    int stencil = 0, Q = 9, D = 2;
    int64_t dims[3] = {1, 1, 1};
    int64_t N = 0, plane = 0;
    double tau = 1.0, omega = 1.0;
    int coll = LB_BGK;
    double relax[3] = {0.25, 0.0, 0.0};  // lb_set_relaxation values (TRT: Lambda; MRT: three tau_g)
    lb_options opt{};
    int device = 0;
    int sms = 0;  // multiprocessors of the device
    cudaStream_t stream = nullptr;
    lb::Geom g{};

    void* ab[2] = {nullptr, nullptr};  // AB ping-pong buffers (AA uses ab[0])
    void* state = nullptr;             // buffer holding the current state
    int aa_parity = 0;                 // AA: 0 natural (even), 1 odd
    void* F = nullptr;                 // force [D][plane], arithmetic type
    void* links = nullptr;             // bounce-back links [plane] (uint32), see lb::Geom
    void* wall_u = nullptr;            // wall velocity [D][plane], arithmetic type
    std::vector<double> net;           // learned network (805 or 545 values), passed to kernels by value
    void* tc_table = nullptr;          // learned_tc: packed BF16 weight fragments on the device
    void* x3_table = nullptr;          // learned, FP32 arithmetic: split BF16 weight fragments (device)
    unsigned* status = nullptr;
    double* partials = nullptr;
    int64_t partials_cap = 0;
    double* dsmall = nullptr;          // device scratch for small results (8 doubles)
    int64_t steps = 0;
    int64_t launches = 0;
    bool failed = false;

    // recording for the adjoint
    bool recording = false;
    std::vector<void*> ckpt;   // ckpt[s] represents f^{s k}
    std::vector<void*> ring;   // k - 1 recompute buffers
    void* lam[2] = {nullptr, nullptr};
    void* gF = nullptr;        // force-gradient accumulator [D][plane]
    void* gtheta = nullptr;    // learned: per-block parameter gradient partials
    int64_t gtheta_cap = 0;    // bytes

    // spectral flow control (Sec. 3.2): every step collides at u + du, du = -kappa grad_u R
    bool sc_on = false;
    int sc_logn = 0;
    double sc_cutoff = 2e-5, sc_kappa = 5e-5;
    void* sc_spec = nullptr;     // [n][n] complex values of the arithmetic type, then the tables (spectral_layout)
    double* sc_small = nullptr;  // partials [n/2][<= n], sigma, grad, r2 [n/2 each], cost [1], sigma0, l0 [n/2 each]
    void* sc_du = nullptr;       // [2][plane] arithmetic type

    // CUDA graph of a two-step cycle, replayed by lb_step when nothing is recorded
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t cycle = nullptr;
    void* cycle_state = nullptr;  // state buffer the cycle starts from (and returns to)
    int64_t cycle_launches = 0;   // kernel launches one replay of the cycle makes
    bool graphs = true;
};

namespace {

bool is_learned(int coll) { return coll == LB_LEARNED_MRT || coll == LB_LEARNED_MRT3; }
// trained parameters of the context's network (the parameter-gradient length)
int net_theta(int coll) { return coll == LB_LEARNED_MRT3 ? lb::kNet3Theta : lb::kNetTheta; }

int64_t pop_bytes(const lb_ctx* c) { return (int64_t)c->Q * c->plane * storage_bytes(c->opt.storage); }
int64_t real_pop_bytes(const lb_ctx* c) { return (int64_t)c->Q * c->plane * real_bytes(c->opt.storage); }

lb_status cuda_fail(lb_ctx* c, cudaError_t e, const char* what)
{
    if (c) c->failed = true;
    return fail(LB_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define LB_CUDA(ctx, call, what)                                  \
    do {                                                          \
        cudaError_t _e = (call);                                  \
        if (_e != cudaSuccess) return cuda_fail((ctx), _e, what); \
    } while (0)

lb_status alloc(lb_ctx* c, void** p, int64_t bytes, const char* what)
{
    cudaError_t e = cudaMalloc(p, (size_t)bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return fail(LB_ERR_OOM, "allocating %lld bytes for %s: %s", (long long)bytes, what, cudaGetErrorString(e));
    }
    (void)c;
    return LB_OK;
}

bool mem_host(lb_mem m) { return m == LB_HOST_F64 || m == LB_HOST_F32; }
int mem_f64(lb_mem m) { return (m == LB_HOST_F64 || m == LB_DEVICE_F64) ? 1 : 0; }
bool mem_valid(int m) { return m >= 0 && m <= 3; }

lb_status check_ctx(const lb_ctx* c)
{
    if (!c) return fail(LB_ERR_ARG, "null context");
    if (c->failed) return fail(LB_ERR_STATE, "context failed after an earlier CUDA error");
    return LB_OK;
}

lb::OpArgs base_args(lb_ctx* c, int op)
{
    lb::OpArgs a;
    a.op = op;
    a.storage = c->opt.storage;
    a.coll = c->coll;
    a.force = c->F != nullptr && c->coll != LB_NONE;
    a.mode = c->opt.layout == LB_LAYOUT_AB ? lb::AB : (c->aa_parity ? lb::AA_ODD : lb::AA_EVEN);
    a.src = c->state;
    a.F = c->F;
    a.g = c->g;
    a.omega = c->omega;
    a.npt = c->opt.nodes_per_thread;
    a.sms = c->sms;
    if (c->coll == LB_TRT) {
        a.rx[0] = 1.0 / (0.5 + c->relax[0] / (c->tau - 0.5));  // 1 / tau_minus
    } else if (c->coll == LB_KBC) {
        a.rx[0] = 2.0 * c->tau;  // 1 / beta
    } else if (c->coll == LB_MRT) {
        for (int k = 0; k < 3; ++k) a.rx[k] = 1.0 / c->relax[k];
    }
    a.status = c->status;
    a.stream = c->stream;
    a.tc_table = c->tc_table;
    a.x3_table = c->x3_table;
    return a;
}

// Byte offsets in c->sc_spec of the spectral-control tables after the complex field [n][n]:
// level twiddles, the shell of every mode [n][n] int16, the first |ky| of every shell per
// column [n/2 + 1][n/2 + 1] int16 (each 256-byte aligned); *total = the allocation's size.
struct SpectralLayout {
    size_t tw, shell, first, total;
};
static SpectralLayout spectral_layout(int64_t n, int storage)
{
    auto up = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t cx = 2 * real_bytes(storage), K = (size_t)n / 2;
    SpectralLayout l;
    l.tw = up((size_t)n * n * cx);
    l.shell = l.tw + up(lb::spectral_twiddle_count((int)n) * cx);
    l.first = l.shell + up((size_t)n * n * 2);
    l.total = l.first + up((K + 1) * (K + 1) * 2);
    return l;
}

// spectral-control scratch views of c->sc_spec and c->sc_small
lb::SpectralArgs spectral_args(lb_ctx* c, const lb::OpArgs& a)
{
    lb::SpectralArgs s;
    s.a = a;
    s.n = (int)c->dims[0];
    s.logn = c->sc_logn;
    s.spec = c->sc_spec;
    if (c->sc_spec) {
        const SpectralLayout l = spectral_layout(s.n, c->opt.storage);
        s.tw = (const char*)c->sc_spec + l.tw;
        s.shell = (const char*)c->sc_spec + l.shell;
        s.first = (const char*)c->sc_spec + l.first;
    }
    const int64_t K = s.n / 2;
    s.partials = c->sc_small;
    s.sigma = s.partials + (int64_t)s.n * K;
    s.grad = s.sigma + K;
    s.r2 = s.grad + K;
    s.cost = s.r2 + K;
    s.sigma0 = c->sc_on ? s.cost + 1 : nullptr;
    s.l0 = c->sc_on ? s.cost + 1 + K : nullptr;
    s.cutoff = c->sc_cutoff;
    s.kappa = c->sc_kappa;
    s.du = c->sc_on ? c->sc_du : nullptr;
    return s;
}

lb_status launch(lb_ctx* c, const lb::OpArgs& a, const char* what)
{
    cudaError_t e;
    if (c->sc_on && a.op == lb::OP_UPDATE) {
        // spectral flow control: du from the state and the step at u + du
        int n = 0;
        e = lb::spectral_step(spectral_args(c, a), &n);
        c->launches += n;
        if (e != cudaSuccess) return cuda_fail(c, e, what);
        return LB_OK;
    }
    if (a.coll == LB_LEARNED_MRT && (a.op == lb::OP_UPDATE || a.op == lb::OP_ADJ_STEP))
        e = lb::run_learned_d2q9(a, c->net.data(), a.op == lb::OP_UPDATE && c->opt.learned_tc);
    else if (a.coll == LB_LEARNED_MRT3 && (a.op == lb::OP_UPDATE || a.op == lb::OP_ADJ_STEP))
        e = lb::run_learned3_d2q9(a, c->net.data(), a.op == lb::OP_UPDATE && c->opt.learned_tc);
    else
        e = lb::run_op(c->stencil, a);
    c->launches += 1;
    if (e != cudaSuccess) return cuda_fail(c, e, what);
    return LB_OK;
}

// Staging of caller arrays: device arrays are used in place; host arrays are
// copied through a stream-ordered temporary device buffer.
struct Staged {
    lb_ctx* c = nullptr;
    void* dev = nullptr;
    void* tmp = nullptr;
    bool direct = false;  // a page-locked host array the kernels use in place
    int64_t bytes = 0;
    ~Staged()
    {
        if (tmp) cudaFreeAsync(tmp, c->stream);
    }
};

// The device address of a page-locked (pinned or registered) host array, or null for pageable
// memory. Kernels read and write such arrays in place (over the host link: NVLink-C2C on
// Grace-Blackwell), which saves the staging buffer and its copy; pageable arrays are staged.
static void* host_direct(const void* p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

lb_status stage_in(lb_ctx* c, Staged& s, const void* p, int64_t count, lb_mem m, const char* what)
{
    s.c = c;
    s.bytes = count * (mem_f64(m) ? 8 : 4);
    if (!mem_host(m)) {
        s.dev = const_cast<void*>(p);
        return LB_OK;
    }
    if (void* d = host_direct(p)) {  // read once by the call's kernels
        s.dev = d;
        s.direct = true;
        return LB_OK;
    }
    cudaError_t e = cudaMallocAsync(&s.tmp, (size_t)s.bytes, c->stream);
    if (e != cudaSuccess) {
        s.tmp = nullptr;
        cudaGetLastError();
        return fail(LB_ERR_OOM, "staging %s: %s", what, cudaGetErrorString(e));
    }
    LB_CUDA(c, cudaMemcpyAsync(s.tmp, p, (size_t)s.bytes, cudaMemcpyHostToDevice, c->stream), what);
    s.dev = s.tmp;
    return LB_OK;
}

lb_status stage_out_alloc(lb_ctx* c, Staged& s, void* p, int64_t count, lb_mem m, bool copy_in, const char* what)
{
    s.c = c;
    s.bytes = count * (mem_f64(m) ? 8 : 4);
    if (!mem_host(m)) {
        s.dev = p;
        return LB_OK;
    }
    // a pure output (written once per element) goes straight to page-locked host memory; an
    // accumulator (copy_in) is staged, since its kernels add to it on every step
    if (void* d = copy_in ? nullptr : host_direct(p)) {
        s.dev = d;
        s.direct = true;
        return LB_OK;
    }
    cudaError_t e = cudaMallocAsync(&s.tmp, (size_t)s.bytes, c->stream);
    if (e != cudaSuccess) {
        s.tmp = nullptr;
        cudaGetLastError();
        return fail(LB_ERR_OOM, "staging %s: %s", what, cudaGetErrorString(e));
    }
    if (copy_in) LB_CUDA(c, cudaMemcpyAsync(s.tmp, p, (size_t)s.bytes, cudaMemcpyHostToDevice, c->stream), what);
    s.dev = s.tmp;
    return LB_OK;
}

lb_status stage_out_finish(lb_ctx* c, Staged& s, void* p, const char* what)
{
    if (s.direct) {  // written in place: ready once the stream has run
        LB_CUDA(c, cudaStreamSynchronize(c->stream), what);
        return LB_OK;
    }
    if (!s.tmp) return LB_OK;
    LB_CUDA(c, cudaMemcpyAsync(p, s.tmp, (size_t)s.bytes, cudaMemcpyDeviceToHost, c->stream), what);
    LB_CUDA(c, cudaStreamSynchronize(c->stream), what);
    return LB_OK;
}

lb_status ensure_partials(lb_ctx* c, int64_t count)
{
    if (c->partials_cap >= count) return LB_OK;
    if (c->partials) cudaFree(c->partials);
    c->partials = nullptr;
    c->partials_cap = 0;
    lb_status s = alloc(c, (void**)&c->partials, count * 8, "reduction partials");
    if (s == LB_OK) c->partials_cap = count;
    return s;
}

void drop_cycle(lb_ctx* c)
{
    if (c->cycle) cudaGraphExecDestroy(c->cycle);
    c->cycle = nullptr;
    c->cycle_state = nullptr;
}

void reset_recording(lb_ctx* c)
{
    c->recording = false;
    c->steps = 0;
}

lb_status record_begin(lb_ctx* c)
{
    if (c->ckpt.empty()) {
        void* p = nullptr;
        lb_status s = alloc(c, &p, pop_bytes(c), "checkpoint");
        if (s != LB_OK) return s;
        c->ckpt.push_back(p);
    }
    LB_CUDA(c, cudaMemcpyAsync(c->ckpt[0], c->state, (size_t)pop_bytes(c), cudaMemcpyDeviceToDevice, c->stream),
            "checkpoint copy");
    c->recording = true;
    return LB_OK;
}

}  // namespace

extern "C" {

void lb_default_options(lb_options* o)
{
    if (!o) return;
    o->storage = LB_F32;
    o->layout = LB_LAYOUT_AB;
    o->cuda_stream = nullptr;
    o->device = -1;
    o->check_every = 0;
    o->record_every = 0;
    o->learned_tc = 0;
    o->graphs = 1;
    o->nodes_per_thread = 0;
}

lb_status lb_create(lb_ctx** out, lb_stencil stencil, const int64_t dims[3], double tau, lb_collision coll,
                    const lb_options* opt)
{
    if (!out) return fail(LB_ERR_ARG, "out is null");
    *out = nullptr;
    if (!dims) return fail(LB_ERR_ARG, "dims is null");
    if ((int)stencil < 0 || (int)stencil > 2) return fail(LB_ERR_ARG, "unknown stencil %d", (int)stencil);
    if ((int)coll < 0 || (int)coll > 7) return fail(LB_ERR_ARG, "unknown collision %d", (int)coll);
    if (!(tau > 0.5) || !std::isfinite(tau)) return fail(LB_ERR_ARG, "tau must be a finite number > 1/2 (got %g)", tau);
    lb_options o;
    lb_default_options(&o);
    if (opt) o = *opt;
    if ((int)o.storage < 0 || (int)o.storage > 3) return fail(LB_ERR_ARG, "unknown storage %d", (int)o.storage);
    if ((int)o.layout < 0 || (int)o.layout > 1) return fail(LB_ERR_ARG, "unknown layout %d", (int)o.layout);
    if (o.check_every < 0 || o.record_every < 0) return fail(LB_ERR_ARG, "negative check_every / record_every");
    if (o.learned_tc != 0 && o.learned_tc != 1) return fail(LB_ERR_ARG, "learned_tc must be 0 or 1");
    if (o.graphs != 0 && o.graphs != 1) return fail(LB_ERR_ARG, "graphs must be 0 or 1");
    if (o.nodes_per_thread != 0 && o.nodes_per_thread != 1 && o.nodes_per_thread != 2 && o.nodes_per_thread != 4)
        return fail(LB_ERR_ARG, "nodes_per_thread must be 0, 1, 2 or 4");
    if (o.learned_tc && (!is_learned(coll) || o.storage == LB_F64))
        return fail(LB_ERR_UNSUPPORTED, "learned_tc needs a learned collision with FP32 or half storage");
    if (o.learned_tc && 9 * ((dims[0] * dims[1] * dims[2] + 63) / 64 * 64) > (int64_t)0x7FFFFFFF)
        return fail(LB_ERR_UNSUPPORTED, "learned_tc addresses the populations with 32-bit offsets: 9 x plane must stay below 2^31");
    const int D = stencil == LB_D2Q9 ? 2 : 3;
    for (int a = 0; a < 3; ++a)
        if (dims[a] < 1 || dims[a] > 65535) return fail(LB_ERR_ARG, "dims[%d] = %lld out of [1, 65535]", a, (long long)dims[a]);
    if (D == 2 && dims[2] != 1) return fail(LB_ERR_ARG, "2D stencil needs dims[2] == 1");
    const int64_t N = dims[0] * dims[1] * dims[2];
    if (N >= ((int64_t)1 << 31)) return fail(LB_ERR_ARG, "grid of %lld nodes exceeds 2^31 - 1", (long long)N);
    if (is_learned(coll) && stencil != LB_D2Q9)
        return fail(LB_ERR_UNSUPPORTED, "the learned collision is defined for D2Q9 only");
    if (coll == LB_MRT && stencil != LB_D2Q9) return fail(LB_ERR_UNSUPPORTED, "MRT is provided for D2Q9 only");
    if (coll == LB_KBC && stencil == LB_D3Q19)
        return fail(LB_ERR_UNSUPPORTED, "KBC needs a tensor-product velocity set (D2Q9 or D3Q27)");
    if (o.record_every > 0 && o.layout != LB_LAYOUT_AB)
        return fail(LB_ERR_UNSUPPORTED, "recording for the adjoint needs the AB layout");
    if (o.record_every > 0 && (coll == LB_TRT || coll == LB_KBC || coll == LB_MRT))
        return fail(LB_ERR_UNSUPPORTED, "no adjoint of the TRT, KBC or MRT collision");

    int dev = o.device;
    if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) return fail(LB_ERR_CUDA, "no CUDA device");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || dev >= ndev) return fail(LB_ERR_ARG, "bad device %d", dev);
    DeviceGuard guard(dev);
    if (!guard.ok) return fail(LB_ERR_CUDA, "cannot select device %d", dev);

    lb_ctx* c = new lb_ctx();
    c->stencil = stencil;
    c->Q = stencil == LB_D2Q9 ? 9 : (stencil == LB_D3Q19 ? 19 : 27);
    c->D = D;
    for (int a = 0; a < 3; ++a) c->dims[a] = dims[a];
    c->N = N;
    // pad each population plane to a multiple of 64 elements (128 B for half, 512 B for FP64)
    c->plane = (N + 63) / 64 * 64;
    c->tau = tau;
    c->omega = 1.0 / tau;
    c->coll = coll;
    if (coll == LB_MRT) c->relax[0] = c->relax[1] = c->relax[2] = 1.0;
    c->opt = o;
    c->device = dev;
    if (cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) c->sms = 0;
    c->stream = (cudaStream_t)o.cuda_stream;
    c->g.nx = (int)dims[0];
    c->g.ny = (int)dims[1];
    c->g.nz = (int)dims[2];
    c->g.plane = c->plane;

    lb_status s = LB_OK;
    const int nbuf = o.layout == LB_LAYOUT_AB ? 2 : 1;
    for (int b = 0; b < nbuf && s == LB_OK; ++b) s = alloc(c, &c->ab[b], pop_bytes(c), "population buffer");
    if (s == LB_OK) s = alloc(c, (void**)&c->status, 64, "status word");
    if (s == LB_OK) s = alloc(c, (void**)&c->dsmall, 64, "small results");
    if (s != LB_OK) {
        lb_destroy(c);
        return s;
    }
    c->state = c->ab[0];
    cudaError_t e = cudaSuccess;
    for (int b = 0; b < nbuf && e == cudaSuccess; ++b) e = cudaMemsetAsync(c->ab[b], 0, (size_t)pop_bytes(c), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->status, 0, 64, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        lb_destroy(c);
        return fail(LB_ERR_CUDA, "initialising buffers: %s", cudaGetErrorString(e));
    }
    *out = c;
    return LB_OK;
}

void lb_destroy(lb_ctx* c)
{
    if (!c) return;
    DeviceGuard guard(c->device);
    cudaStreamSynchronize(c->stream);
    if (c->cycle) cudaGraphExecDestroy(c->cycle);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    void* ptrs[] = {c->ab[0], c->ab[1], c->F, c->tc_table, c->x3_table, c->status, c->partials, c->dsmall,
                    c->lam[0], c->lam[1], c->gF, c->gtheta, c->links, c->wall_u, c->sc_spec, c->sc_small, c->sc_du};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    for (void* p : c->ckpt)
        if (p) cudaFree(p);
    for (void* p : c->ring)
        if (p) cudaFree(p);
    delete c;
}

lb_status lb_init_from_moments(lb_ctx* c, const void* rho, const void* u, lb_mem m)
{
    lb_status s = check_ctx(c);
    if (s != LB_OK) return s;
    if (!rho || !u || !mem_valid(m)) return fail(LB_ERR_ARG, "rho, u and a valid lb_mem are required");
    DeviceGuard guard(c->device);
    Staged sr, su;
    if ((s = stage_in(c, sr, rho, c->N, m, "rho")) != LB_OK) return s;
    if ((s = stage_in(c, su, u, c->N * c->D, m, "u")) != LB_OK) return s;
    c->aa_parity = 0;
    c->state = c->ab[0];
    lb::OpArgs a = base_args(c, lb::OP_INIT_EQ);
    a.dst = c->state;
    a.in0 = sr.dev;
    a.in1 = su.dev;
    a.io_f64 = mem_f64(m);
    if ((s = launch(c, a, "init_eq")) != LB_OK) return s;
    reset_recording(c);
    return LB_OK;
}

lb_status lb_set_force(lb_ctx* c, const void* F, lb_mem m)
{
    lb_status s = check_ctx(c);
    if (s != LB_OK) return s;
    drop_cycle(c);  // the force pointer (or its absence) is baked into the captured steps
    if (!mem_valid(m)) return fail(LB_ERR_ARG, "invalid lb_mem");
    if (F && (is_learned(c->coll) || c->coll == LB_KBC || c->coll == LB_MRT))
        return fail(LB_ERR_UNSUPPORTED, "the learned, KBC and MRT collisions take no force");
    if (F && c->sc_on) return fail(LB_ERR_UNSUPPORTED, "spectral flow control takes no body force");
    DeviceGuard guard(c->device);
    if (!F) {
        if (c->F) {
            cudaStreamSynchronize(c->stream);
            cudaFree(c->F);
        }
        c->F = nullptr;
        return LB_OK;
    }
    if (!c->F) {
        const int64_t bytes = (int64_t)c->D * c->plane * real_bytes(c->opt.storage);
        if ((s = alloc(c, &c->F, bytes, "force")) != LB_OK) return s;
        LB_CUDA(c, cudaMemsetAsync(c->F, 0, (size_t)bytes, c->stream), "force clear");
    }
    Staged sf;
    if ((s = stage_in(c, sf, F, c->N * c->D, m, "force")) != LB_OK) return s;
    LB_CUDA(c, lb::convert_copy(sf.dev, mem_f64(m), c->F, c->opt.storage == LB_F64, c->N, c->N, c->plane, c->D, 0,
                                c->stream),
            "force copy");
    c->launches += 1;
    return LB_OK;
}

lb_status lb_set_mlp(lb_ctx* c, const void* params, int64_t n, lb_mem m)
{
    lb_status s = check_ctx(c);
    if (s != LB_OK) return s;
    if (!is_learned(c->coll)) return fail(LB_ERR_STATE, "context does not use a learned collision");
    const int want = c->coll == LB_LEARNED_MRT3 ? lb::kNet3Values : lb::kNetValues;
    if (!params || n != want || !mem_valid(m))
        return fail(LB_ERR_ARG, "need %d network values (got %lld)", want, (long long)n);
    DeviceGuard guard(c->device);
    const int f64 = mem_f64(m);
    std::vector<unsigned char> tmp((size_t)n * (f64 ? 8 : 4));
    if (mem_host(m)) {
        std::memcpy(tmp.data(), params, tmp.size());
    } else {
        // the values are passed to the kernels by value, so they come to the host
        LB_CUDA(c, cudaMemcpyAsync(tmp.data(), params, tmp.size(), cudaMemcpyDeviceToHost, c->stream), "network read");
        LB_CUDA(c, cudaStreamSynchronize(c->stream), "network read");
    }
    std::vector<double> v((size_t)n);
    for (int64_t k = 0; k < n; ++k)
        v[(size_t)k] = f64 ? ((const double*)tmp.data())[k] : (double)((const float*)tmp.data())[k];
    for (double x : v)
        if (!std::isfinite(x)) return fail(LB_ERR_ARG, "network values must be finite");
    if (c->opt.learned_tc) {
        const bool three = c->coll == LB_LEARNED_MRT3;
        const size_t bytes = three ? lb::learned3_tc_table_bytes() : lb::learned_tc_table_bytes();
        if (!c->tc_table && (s = alloc(c, &c->tc_table, (int64_t)bytes, "tensor-core weight table")) != LB_OK) return s;
        std::vector<unsigned char> tab(bytes);
        if (three) lb::learned3_tc_pack(v.data(), tab.data());
        else lb::learned_tc_pack(v.data(), tab.data());
        // the previous table may still be read by queued steps: order the copy on the stream
        LB_CUDA(c, cudaMemcpyAsync(c->tc_table, tab.data(), bytes, cudaMemcpyHostToDevice, c->stream), "weight table");
        LB_CUDA(c, cudaStreamSynchronize(c->stream), "weight table");
    }
    if (c->opt.storage != LB_F64) {
        // the FP32 arithmetic's tensor-core kernels read the weights split into BF16 terms
        const bool three = c->coll == LB_LEARNED_MRT3;
        const size_t bytes = lb::learned_x3_table_bytes(three);
        if (!c->x3_table && (s = alloc(c, &c->x3_table, (int64_t)bytes, "split weight table")) != LB_OK) return s;
        std::vector<unsigned char> tab(bytes);
        lb::learned_x3_pack(v.data(), three, tab.data());
        LB_CUDA(c, cudaMemcpyAsync(c->x3_table, tab.data(), bytes, cudaMemcpyHostToDevice, c->stream), "weight table");
        LB_CUDA(c, cudaStreamSynchronize(c->stream), "weight table");
    }
    c->net.swap(v);
    drop_cycle(c);  // the network is a by-value kernel argument of the captured steps
    return LB_OK;
}

lb_status lb_set_solid(lb_ctx* c, const void* mask, const void* wall_u, lb_mem m)
{
    lb_status s = check_ctx(c);
    if (s != LB_OK) return s;
    if (!mem_valid(m)) return fail(LB_ERR_ARG, "invalid lb_mem");
    if (!mask && wall_u) return fail(LB_ERR_ARG, "a wall velocity needs a mask");
    if (mask) {
        if (c->opt.layout != LB_LAYOUT_AB) return fail(LB_ERR_UNSUPPORTED, "walls need the AB layout");
        if (is_learned(c->coll)) return fail(LB_ERR_UNSUPPORTED, "the learned collisions have no walls");
        if (c->sc_on) return fail(LB_ERR_UNSUPPORTED, "spectral flow control needs a periodic grid without walls");
        if (c->opt.record_every > 0) return fail(LB_ERR_UNSUPPORTED, "no adjoint with walls");
    }
    DeviceGuard guard(c->device);
    drop_cycle(c);  // the link table is a by-value kernel argument of the captured steps
    // With walls the buffer holds reflected values in the slots of solid nodes, so a node
    // that turns fluid would pull stale values. Replacing walls therefore keeps the exposed
    // state (solid nodes at rest) and writes it back under the new geometry.
    void* keep = nullptr;
    if (c->links) {
        cudaError_t e = cudaMallocAsync(&keep, (size_t)(c->Q * c->N * 8), c->stream);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(LB_ERR_OOM, "keeping the state across the wall change: %s", cudaGetErrorString(e));
        }
        lb::OpArgs a = base_args(c, lb::OP_GET);
        a.out0 = keep;
        a.io_f64 = 1;
        if ((s = launch(c, a, "keep state")) != LB_OK) return s;
    }
    auto restore = [&]() -> lb_status {
        if (!keep) return LB_OK;
        lb::OpArgs a = base_args(c, lb::OP_SET);
        a.dst = c->state;
        a.in0 = keep;
        a.io_f64 = 1;
        lb_status r = launch(c, a, "restore state");
        cudaFreeAsync(keep, c->stream);
        keep = nullptr;
        return r;
    };
    if (!mask) {
        c->g.links = nullptr;
        c->g.wall_u = nullptr;
        if ((s = restore()) != LB_OK) return s;
        cudaStreamSynchronize(c->stream);
        if (c->links) cudaFree(c->links);
        if (c->wall_u) cudaFree(c->wall_u);
        c->links = c->wall_u = nullptr;
        return LB_OK;
    }
    if (!c->links && (s = alloc(c, &c->links, c->plane * 4, "bounce-back links")) != LB_OK) return s;
    // the mask: N bytes, on the host or the device as mem says
    const void* dmask = mask;
    void* tmp = nullptr;
    if (mem_host(m)) {
        cudaError_t e = cudaMallocAsync(&tmp, (size_t)c->N, c->stream);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(LB_ERR_OOM, "staging the mask: %s", cudaGetErrorString(e));
        }
        LB_CUDA(c, cudaMemcpyAsync(tmp, mask, (size_t)c->N, cudaMemcpyHostToDevice, c->stream), "mask copy");
        dmask = tmp;
    }
    lb::OpArgs a = base_args(c, lb::OP_LINKS);
    a.mode = lb::AB;
    a.in0 = dmask;
    a.out0 = c->links;
    s = launch(c, a, "bounce-back links");
    if (tmp) cudaFreeAsync(tmp, c->stream);
    if (s != LB_OK) return s;
    if (wall_u) {
        const int64_t bytes = (int64_t)c->D * c->plane * real_bytes(c->opt.storage);
        if (!c->wall_u && (s = alloc(c, &c->wall_u, bytes, "wall velocity")) != LB_OK) return s;
        LB_CUDA(c, cudaMemsetAsync(c->wall_u, 0, (size_t)bytes, c->stream), "wall velocity clear");
        Staged sw;
        if ((s = stage_in(c, sw, wall_u, c->N * c->D, m, "wall velocity")) != LB_OK) return s;
        LB_CUDA(c, lb::convert_copy(sw.dev, mem_f64(m), c->wall_u, c->opt.storage == LB_F64, c->N, c->N, c->plane,
                                    c->D, 0, c->stream),
                "wall velocity copy");
        c->launches += 1;
    } else if (c->wall_u) {
        cudaStreamSynchronize(c->stream);
        cudaFree(c->wall_u);
        c->wall_u = nullptr;
    }
    c->g.links = (const unsigned*)c->links;
    c->g.wall_u = c->wall_u;
    return restore();
}

lb_status lb_set_relaxation(lb_ctx* c, const double* params, int n)
{
    lb_status s = check_ctx(c);
    if (s != LB_OK) return s;
    if (c->coll != LB_TRT && c->coll != LB_MRT)
        return fail(LB_ERR_STATE, "only the TRT and MRT collisions take further relaxation parameters");
    const int need = c->coll == LB_TRT ? 1 : 3;
    if (!params || n != need) return fail(LB_ERR_ARG, "need %d value(s), got %d", need, n);
    for (int k = 0; k < n; ++k) {
        if (!std::isfinite(params[k])) return fail(LB_ERR_ARG, "relaxation parameters must be finite");
        if (c->coll == LB_TRT && !(params[k] > 0.0)) return fail(LB_ERR_ARG, "Lambda must be > 0");
        if (c->coll == LB_MRT && !(params[k] > 0.5)) return fail(LB_ERR_ARG, "relaxation times must be > 1/2");
    }
    for (int k = 0; k < n; ++k) c->relax[k] = params[k];
    drop_cycle(c);  // the rates are by-value kernel arguments of the captured steps
    return LB_OK;
}

// Grid edge n and log2(n) of a context the spectral calls accept (square D2Q9, n = 2^k).
static lb_status spectral_grid(const lb_ctx* c, int* logn)
{
    if (c->stencil != LB_D2Q9) return fail(LB_ERR_UNSUPPORTED, "the spectral calls are defined for D2Q9");
    const int64_t n = c->dims[0];
    if (c->dims[1] != n || n < 4 || n > lb::kSpecMaxN || (n & (n - 1)))
        return fail(LB_ERR_UNSUPPORTED, "the spectral calls need a square grid of 2^k nodes per side, 4 <= n <= %d",
                    lb::kSpecMaxN);
    int l = 0;
    while ((int64_t(1) << l) < n) ++l;
    *logn = l;
    return LB_OK;
}

static lb_status spectral_alloc(lb_ctx* c)
{
    const int64_t n = c->dims[0], K = n / 2;
    lb_status s;
    if (!c->sc_spec) {
        // the complex field [n][n], then the tables of the line transforms (computed here, once)
        const SpectralLayout l = spectral_layout(n, c->opt.storage);
        if ((s = alloc(c, &c->sc_spec, l.total, "spectrum")) != LB_OK) return s;
        char* base = (char*)c->sc_spec;
        int nl = 0;
        LB_CUDA(c, lb::spectral_tables(base + l.tw, base + l.shell, base + l.first, (int)n, c->opt.storage, c->stream,
                                       &nl),
                "spectral tables");
        c->launches += nl;
    }
    if (!c->sc_small && (s = alloc(c, (void**)&c->sc_small, (n * K + 5 * K + 1) * 8, "spectral sums")) != LB_OK)
        return s;
    return LB_OK;
}

lb_status lb_set_spectral_control(lb_ctx* c, const double* sigma0, int64_t K, double cutoff, double kappa)
{
    lb_status s = check_ctx(c);
    if (s != LB_OK) return s;
    if (!sigma0) {
        c->sc_on = false;
        drop_cycle(c);
        return LB_OK;
    }
    int logn = 0;
    if ((s = spectral_grid(c, &logn)) != LB_OK) return s;
    if (c->coll != LB_BGK) return fail(LB_ERR_UNSUPPORTED, "spectral flow control is defined with the BGK collision");
    if (c->F) return fail(LB_ERR_UNSUPPORTED, "spectral flow control takes no body force");
    if (c->links) return fail(LB_ERR_UNSUPPORTED, "spectral flow control needs a periodic grid without walls");
    if (c->opt.record_every > 0) return fail(LB_ERR_UNSUPPORTED, "no adjoint of the spectral flow control");
    if (K != c->dims[0] / 2) return fail(LB_ERR_ARG, "sigma0 needs n/2 = %lld shells", (long long)(c->dims[0] / 2));
    if (!(cutoff > 0.0) || !std::isfinite(cutoff) || !(kappa >= 0.0) || !std::isfinite(kappa))
        return fail(LB_ERR_ARG, "cutoff must be > 0 and kappa >= 0, both finite");
    for (int64_t k = 0; k < K; ++k)
        if (!(sigma0[k] >= 0.0) || !std::isfinite(sigma0[k])) return fail(LB_ERR_ARG, "sigma0 must be finite and >= 0");
    DeviceGuard guard(c->device);
    if ((s = spectral_alloc(c)) != LB_OK) return s;
    if (!c->sc_du && (s = alloc(c, &c->sc_du, 2 * c->plane * real_bytes(c->opt.storage), "velocity shift")) != LB_OK)
        return s;
    const int64_t n = c->dims[0];
    // sigma0 and ln max(sigma0, cutoff) sit after partials, sigma, grad, r2 and cost; ordered on
    // the stream after queued steps
    std::vector<double> target((size_t)(2 * K));
    for (int64_t k = 0; k < K; ++k) {
        target[(size_t)k] = sigma0[k];
        target[(size_t)(K + k)] = std::log(std::fmax(sigma0[k], cutoff));
    }
    LB_CUDA(c, cudaMemcpyAsync(c->sc_small + n * K + 3 * K + 1, target.data(), (size_t)(2 * K) * 8,
                               cudaMemcpyHostToDevice, c->stream),
            "sigma0 copy");
    LB_CUDA(c, cudaStreamSynchronize(c->stream), "sigma0 copy");
    c->sc_on = true;
    c->sc_logn = logn;
    c->sc_cutoff = cutoff;
    c->sc_kappa = kappa;
    drop_cycle(c);  // the captured steps change
    return LB_OK;
}

lb_status lb_spectrum(lb_ctx* c, double* sigma, double* cost)
{
    lb_status s = check_ctx(c);
    if (s != LB_OK) return s;
    if (!sigma && !cost) return fail(LB_ERR_ARG, "sigma or cost is required");
    if (cost && !c->sc_on) return fail(LB_ERR_STATE, "the cost needs a target (lb_set_spectral_control)");
    int logn = 0;
    if ((s = spectral_grid(c, &logn)) != LB_OK) return s;
    DeviceGuard guard(c->device);
    if ((s = spectral_alloc(c)) != LB_OK) return s;
    c->sc_logn = logn;
    lb::SpectralArgs sa = spectral_args(c, base_args(c, lb::OP_MOMENTS));
    sa.du = nullptr;
    int n = 0;
    cudaError_t e = lb::spectral_shift(sa, &n);
    c->launches += n;
    if (e != cudaSuccess) return cuda_fail(c, e, "spectrum");
    const int64_t K = c->dims[0] / 2;
    if (sigma) LB_CUDA(c, cudaMemcpyAsync(sigma, sa.sigma, (size_t)K * 8, cudaMemcpyDeviceToHost, c->stream), "sigma");
    if (cost) LB_CUDA(c, cudaMemcpyAsync(cost, sa.cost, 8, cudaMemcpyDeviceToHost, c->stream), "cost");
    LB_CUDA(c, cudaStreamSynchronize(c->stream), "spectrum sync");
    return LB_OK;
}

lb_status lb_spectral_shift(lb_ctx* c, void* du, lb_mem m)
{
    lb_status s = check_ctx(c);
    if (s != LB_OK) return s;
    if (!du || !mem_valid(m)) return fail(LB_ERR_ARG, "du and a valid lb_mem are required");
    if (!c->sc_on) return fail(LB_ERR_STATE, "spectral flow control is not set");
    DeviceGuard guard(c->device);
    lb::SpectralArgs sa = spectral_args(c, base_args(c, lb::OP_MOMENTS));
    int n = 0;
    cudaError_t e = lb::spectral_shift(sa, &n);
    c->launches += n;
    if (e != cudaSuccess) return cuda_fail(c, e, "velocity shift");
    Staged so;
    if ((s = stage_out_alloc(c, so, du, c->N * c->D, m, false, "du")) != LB_OK) return s;
    LB_CUDA(c, lb::convert_copy(c->sc_du, c->opt.storage == LB_F64, so.dev, mem_f64(m), c->N, c->plane, c->N, c->D, 0,
                                c->stream),
            "du copy");
    c->launches += 1;
    return stage_out_finish(c, so, du, "du");
}

static lb_status step_once(lb_ctx* c)
{
    const int k = c->opt.record_every;
    lb::OpArgs a = base_args(c, lb::OP_UPDATE);
    if (c->opt.layout == LB_LAYOUT_AA) {
        a.dst = c->state;
        lb_status s = launch(c, a, "stream-collide (AA)");
        if (s != LB_OK) return s;
        c->aa_parity ^= 1;
        c->steps += 1;
        return LB_OK;
    }
    void* dst = (c->state == c->ab[0]) ? c->ab[1] : c->ab[0];
    if (k > 0 && (c->steps + 1) % k == 0) {
        const size_t slot = (size_t)((c->steps + 1) / k);
        while (c->ckpt.size() <= slot) {
            void* p = nullptr;
            lb_status s = alloc(c, &p, pop_bytes(c), "checkpoint");
            if (s != LB_OK) return s;
            c->ckpt.push_back(p);
        }
        dst = c->ckpt[slot];
    }
    a.dst = dst;
    lb_status s = launch(c, a, "stream-collide");
    if (s != LB_OK) return s;
    c->state = dst;
    c->steps += 1;
    return LB_OK;
}

lb_status lb_check(lb_ctx* c)
{
    lb_status s = check_ctx(c);
    if (s != LB_OK) return s;
    DeviceGuard guard(c->device);
    unsigned h = 0;
    LB_CUDA(c, cudaMemcpyAsync(&h, c->status, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream), "status read");
    LB_CUDA(c, cudaStreamSynchronize(c->stream), "status sync");
    if (h) {
        LB_CUDA(c, cudaMemsetAsync(c->status, 0, sizeof(unsigned), c->stream), "status clear");
        return fail(LB_ERR_UNSTABLE, "a node had a non-finite or non-positive density");
    }
    return LB_OK;
}

// Capture two consecutive steps (AB: A -> B -> A; AA: even, odd) into a graph on a private
// stream. Returns false (and leaves direct launches in charge) if capture is not possible.
static bool build_cycle(lb_ctx* c)
{
    if (!c->cap_stream && cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        c->cap_stream = nullptr;
        return false;
    }
    drop_cycle(c);
    void* start = c->state;
    const int parity = c->aa_parity;
    const int64_t steps0 = c->steps, launches0 = c->launches;
    cudaStream_t user = c->stream;
    if (cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    c->stream = c->cap_stream;
    bool ok = step_once(c) == LB_OK && step_once(c) == LB_OK;
    c->stream = user;
    const int64_t captured = c->launches - launches0;
    cudaGraph_t graph = nullptr;
    const bool ended = cudaStreamEndCapture(c->cap_stream, &graph) == cudaSuccess;
    // the captured launches did not run: restore the bookkeeping
    c->state = start;
    c->aa_parity = parity;
    c->steps = steps0;
    c->launches = launches0;
    c->failed = false;
    if (!ok || !ended || !graph) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return false;
    }
    cudaGraphExec_t exec = nullptr;
    const bool inst = cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
    cudaGraphDestroy(graph);
    if (!inst) {
        cudaGetLastError();
        return false;
    }
    c->cycle = exec;
    c->cycle_state = start;
    c->cycle_launches = captured;
    return true;
}

lb_status lb_step(lb_ctx* c, int64_t n)
{
    lb_status s = check_ctx(c);
    if (s != LB_OK) return s;
    if (n < 0) return fail(LB_ERR_ARG, "negative step count");
    if (is_learned(c->coll) && c->net.empty()) return fail(LB_ERR_STATE, "network not set");
    DeviceGuard guard(c->device);
    if (c->opt.record_every > 0 && !c->recording && n > 0)
        if ((s = record_begin(c)) != LB_OK) return s;
    // without recording, pairs of steps replay a captured two-step graph
    const bool use_graph = c->graphs && c->opt.graphs && c->opt.record_every == 0 && n >= 2;
    for (int64_t t = 0; t < n;) {
        const int64_t until_check = c->opt.check_every > 0 ? c->opt.check_every - t % c->opt.check_every : n - t;
        const bool even_start = c->opt.layout == LB_LAYOUT_AB || c->aa_parity == 0;
        if (use_graph && n - t >= 2 && until_check >= 2 && even_start) {
            if (!c->cycle || c->cycle_state != c->state)
                if (!build_cycle(c)) c->graphs = false;
            if (c->cycle) {
                LB_CUDA(c, cudaGraphLaunch(c->cycle, c->stream), "step graph");
                c->steps += 2;
                c->launches += c->cycle_launches;
                t += 2;
                if (c->opt.check_every > 0 && t % c->opt.check_every == 0)
                    if ((s = lb_check(c)) != LB_OK) return s;
                continue;
            }
        }
        if ((s = step_once(c)) != LB_OK) return s;
        ++t;
        if (c->opt.check_every > 0 && t % c->opt.check_every == 0)
            if ((s = lb_check(c)) != LB_OK) return s;
    }
    if (c->opt.check_every > 0 && n % c->opt.check_every != 0) return lb_check(c);
    return LB_OK;
}

lb_status lb_moments(lb_ctx* c, void* rho, void* u, lb_mem m)
{
    lb_status s = check_ctx(c);
    if (s != LB_OK) return s;
    if (!mem_valid(m)) return fail(LB_ERR_ARG, "invalid lb_mem");
    if (!rho && !u) return LB_OK;
    DeviceGuard guard(c->device);
    Staged sr, su;
    if (rho && (s = stage_out_alloc(c, sr, rho, c->N, m, false, "rho")) != LB_OK) return s;
    if (u && (s = stage_out_alloc(c, su, u, c->N * c->D, m, false, "u")) != LB_OK) return s;
    lb::OpArgs a = base_args(c, lb::OP_MOMENTS);
    a.out0 = rho ? sr.dev : nullptr;
    a.out1 = u ? su.dev : nullptr;
    a.io_f64 = mem_f64(m);
    if ((s = launch(c, a, "moments")) != LB_OK) return s;
    if (rho && (s = stage_out_finish(c, sr, rho, "rho")) != LB_OK) return s;
    if (u && (s = stage_out_finish(c, su, u, "u")) != LB_OK) return s;
    return LB_OK;
}

lb_status lb_reduce(lb_ctx* c, double out[6])
{
    lb_status s = check_ctx(c);
    if (s != LB_OK) return s;
    if (!out) return fail(LB_ERR_ARG, "out is null");
    DeviceGuard guard(c->device);
    const int64_t nb = lb::node_grid_blocks(c->g);
    if ((s = ensure_partials(c, 6 * nb)) != LB_OK) return s;
    lb::OpArgs a = base_args(c, lb::OP_REDUCE_PARTIAL);
    a.partials = c->partials;
    if ((s = launch(c, a, "reduce")) != LB_OK) return s;
    LB_CUDA(c, lb::reduce_final(c->partials, nb, 6, c->dsmall, c->stream), "reduce final");
    c->launches += 1;
    double h[6];
    LB_CUDA(c, cudaMemcpyAsync(h, c->dsmall, sizeof(h), cudaMemcpyDeviceToHost, c->stream), "reduce read");
    LB_CUDA(c, cudaStreamSynchronize(c->stream), "reduce sync");
    const double invN = 1.0 / (double)c->N;
    out[0] = h[0];
    out[1] = h[1];
    out[2] = h[2];
    out[3] = h[3];
    out[4] = 0.5 * h[4] * invN;
    out[5] = 0.5 * h[5] * invN;
    return LB_OK;
}

// ------------------------------------------------------------------ slabs
// A context may hold one slab of a larger periodic grid split along its last axis (z in 3D,
// y in 2D), with one ghost layer at each end (local layers 0 and n_last - 1). The populations
// that cross a face are the slots whose velocity has last component +1 or -1.
static int slab_axis(const lb_ctx* c) { return c->D == 3 ? 2 : 1; }
static int64_t slab_layer_nodes(const lb_ctx* c) { return c->D == 3 ? c->dims[0] * c->dims[1] : c->dims[0]; }
static int slab_slots(const lb_ctx* c, int dir, int* slots)
{
    int n = 0;
    for (int i = 0; i < c->Q; ++i) {
        const int cl = c->D == 3 ? lb::c3(i, 2) : lb::c2(i, 1);
        if (cl == dir) slots[n++] = i;
    }
    return n;
}

static lb_status slab_check(lb_ctx* c, int face)
{
    if (face != 0 && face != 1) return fail(LB_ERR_ARG, "face must be 0 (low end) or 1 (high end)");
    if (c->opt.layout != LB_LAYOUT_AB) return fail(LB_ERR_UNSUPPORTED, "the slab exchange needs the AB layout");
    if (c->dims[slab_axis(c)] < 3) return fail(LB_ERR_ARG, "a slab needs two ghost layers and one interior layer");
    return LB_OK;
}

lb_status lb_halo_bytes(const lb_ctx* c, int64_t* bytes)
{
    if (!c) return fail(LB_ERR_ARG, "null context");
    if (!bytes) return fail(LB_ERR_ARG, "bytes is null");
    int slots[27];
    *bytes = (int64_t)slab_slots(c, 1, slots) * slab_layer_nodes(c) * storage_bytes(c->opt.storage);
    return LB_OK;
}

// Copy the crossing populations between the state buffer and buf (device memory): n copies of
// one contiguous layer of one slot each, ordered on the context's stream.
static lb_status slab_copy(lb_ctx* c, int face, void* buf, bool pack)
{
    lb_status s = check_ctx(c);
    if (s != LB_OK) return s;
    if (!buf) return fail(LB_ERR_ARG, "buf is null");
    if ((s = slab_check(c, face)) != LB_OK) return s;
    if (!pack && c->opt.record_every > 0) return fail(LB_ERR_UNSUPPORTED, "no adjoint over slabs");
    DeviceGuard guard(c->device);
    const int64_t nl = c->dims[slab_axis(c)], ln = slab_layer_nodes(c), sb = storage_bytes(c->opt.storage);
    // pack: interior layer next to the face, slots leaving through it; unpack: the face's ghost
    // layer, slots entering through it
    const int dir = pack ? (face == 0 ? -1 : 1) : (face == 0 ? 1 : -1);
    const int64_t layer = pack ? (face == 0 ? 1 : nl - 2) : (face == 0 ? 0 : nl - 1);
    int slots[27];
    const int n = slab_slots(c, dir, slots);
    for (int k = 0; k < n; ++k) {
        char* st = (char*)c->state + ((int64_t)slots[k] * c->plane + layer * ln) * sb;
        char* bf = (char*)buf + (int64_t)k * ln * sb;
        LB_CUDA(c, cudaMemcpyAsync(pack ? bf : st, pack ? st : bf, (size_t)(ln * sb), cudaMemcpyDeviceToDevice, c->stream),
                "halo copy");
    }
    return LB_OK;
}

lb_status lb_halo_pack(lb_ctx* c, int face, void* buf) { return slab_copy(c, face, buf, true); }
lb_status lb_halo_unpack(lb_ctx* c, int face, const void* buf) { return slab_copy(c, face, const_cast<void*>(buf), false); }

lb_status lb_reduce_slab(lb_ctx* c, int64_t first, int64_t count, double out[6])
{
    lb_status s = check_ctx(c);
    if (s != LB_OK) return s;
    if (!out) return fail(LB_ERR_ARG, "out is null");
    const int ax = slab_axis(c);
    if (first < 0 || count < 1 || first + count > c->dims[ax])
        return fail(LB_ERR_ARG, "layers [%lld, %lld) are not inside the last axis", (long long)first,
                    (long long)(first + count));
    DeviceGuard guard(c->device);
    const int64_t nb = lb::node_grid_blocks(c->g);
    if ((s = ensure_partials(c, 6 * nb)) != LB_OK) return s;
    lb::OpArgs a = base_args(c, lb::OP_REDUCE_PARTIAL);
    a.partials = c->partials;
    if ((s = launch(c, a, "reduce")) != LB_OK) return s;
    // the node grid's blocks run x fastest, then y, then z: a layer range is a block range
    const dim3 gr = lb::node_grid(c->g);
    const int64_t per_layer = ax == 2 ? (int64_t)gr.x * gr.y : (int64_t)gr.x;
    LB_CUDA(c, lb::reduce_final(c->partials + 6 * per_layer * first, per_layer * count, 6, c->dsmall, c->stream),
            "reduce final");
    c->launches += 1;
    LB_CUDA(c, cudaMemcpyAsync(out, c->dsmall, 6 * sizeof(double), cudaMemcpyDeviceToHost, c->stream), "reduce read");
    LB_CUDA(c, cudaStreamSynchronize(c->stream), "reduce sync");
    return LB_OK;
}

lb_status lb_get_populations(lb_ctx* c, void* f, lb_mem m)
{
    lb_status s = check_ctx(c);
    if (s != LB_OK) return s;
    if (!f || !mem_valid(m)) return fail(LB_ERR_ARG, "f and a valid lb_mem are required");
    DeviceGuard guard(c->device);
    Staged sf;
    if ((s = stage_out_alloc(c, sf, f, c->N * c->Q, m, false, "populations")) != LB_OK) return s;
    lb::OpArgs a = base_args(c, lb::OP_GET);
    a.out0 = sf.dev;
    a.io_f64 = mem_f64(m);
    if ((s = launch(c, a, "get populations")) != LB_OK) return s;
    return stage_out_finish(c, sf, f, "populations");
}

lb_status lb_set_populations(lb_ctx* c, const void* f, lb_mem m)
{
    lb_status s = check_ctx(c);
    if (s != LB_OK) return s;
    if (!f || !mem_valid(m)) return fail(LB_ERR_ARG, "f and a valid lb_mem are required");
    DeviceGuard guard(c->device);
    Staged sf;
    if ((s = stage_in(c, sf, f, c->N * c->Q, m, "populations")) != LB_OK) return s;
    c->aa_parity = 0;
    c->state = c->ab[0];
    lb::OpArgs a = base_args(c, lb::OP_SET);
    a.dst = c->state;
    a.in0 = sf.dev;
    a.io_f64 = mem_f64(m);
    if ((s = launch(c, a, "set populations")) != LB_OK) return s;
    reset_recording(c);
    return LB_OK;
}

int64_t lb_steps_taken(const lb_ctx* c) { return c ? c->steps : -1; }

lb_status lb_adjoint_seed_moments(lb_ctx* c, const void* grho, const void* gu, void* lam, void* gF, lb_mem m)
{
    lb_status s = check_ctx(c);
    if (s != LB_OK) return s;
    if (!gu || !lam || !mem_valid(m)) return fail(LB_ERR_ARG, "grad_u, lambda and a valid lb_mem are required");
    DeviceGuard guard(c->device);
    Staged sr, su, sl, sg;
    if (grho && (s = stage_in(c, sr, grho, c->N, m, "grad_rho")) != LB_OK) return s;
    if ((s = stage_in(c, su, gu, c->N * c->D, m, "grad_u")) != LB_OK) return s;
    if ((s = stage_out_alloc(c, sl, lam, c->N * c->Q, m, false, "lambda")) != LB_OK) return s;
    const bool want_gF = gF && c->F;
    if (want_gF && (s = stage_out_alloc(c, sg, gF, c->N * c->D, m, true, "grad_F")) != LB_OK) return s;
    lb::OpArgs a = base_args(c, lb::OP_ADJ_SEED);
    a.in0 = grho ? sr.dev : nullptr;
    a.in1 = su.dev;
    a.out0 = sl.dev;
    a.out1 = want_gF ? sg.dev : nullptr;
    a.io_f64 = mem_f64(m);
    if ((s = launch(c, a, "adjoint seed")) != LB_OK) return s;
    if ((s = stage_out_finish(c, sl, lam, "lambda")) != LB_OK) return s;
    if (want_gF && (s = stage_out_finish(c, sg, gF, "grad_F")) != LB_OK) return s;
    return LB_OK;
}

lb_status lb_loss_energy(lb_ctx* c, const void* et, double* loss, void* lam, void* gF, lb_mem m)
{
    lb_status s = check_ctx(c);
    if (s != LB_OK) return s;
    if (!et || !loss || !mem_valid(m)) return fail(LB_ERR_ARG, "e_target, loss and a valid lb_mem are required");
    DeviceGuard guard(c->device);
    Staged se, sl, sg;
    if ((s = stage_in(c, se, et, c->N, m, "e_target")) != LB_OK) return s;
    if (lam && (s = stage_out_alloc(c, sl, lam, c->N * c->Q, m, false, "lambda")) != LB_OK) return s;
    const bool want_gF = gF && c->F;
    if (want_gF && (s = stage_out_alloc(c, sg, gF, c->N * c->D, m, true, "grad_F")) != LB_OK) return s;
    const int64_t nb = lb::node_grid_blocks(c->g);
    if ((s = ensure_partials(c, nb)) != LB_OK) return s;
    lb::OpArgs a = base_args(c, lb::OP_LOSS_ENERGY);
    a.in0 = se.dev;
    a.out0 = lam ? sl.dev : nullptr;
    a.out1 = want_gF ? sg.dev : nullptr;
    a.io_f64 = mem_f64(m);
    a.partials = c->partials;
    if ((s = launch(c, a, "energy loss")) != LB_OK) return s;
    LB_CUDA(c, lb::reduce_final(c->partials, nb, 1, c->dsmall, c->stream), "loss reduce");
    c->launches += 1;
    LB_CUDA(c, cudaMemcpyAsync(loss, c->dsmall, sizeof(double), cudaMemcpyDeviceToHost, c->stream), "loss read");
    LB_CUDA(c, cudaStreamSynchronize(c->stream), "loss sync");
    if (lam && (s = stage_out_finish(c, sl, lam, "lambda")) != LB_OK) return s;
    if (want_gF && (s = stage_out_finish(c, sg, gF, "grad_F")) != LB_OK) return s;
    return LB_OK;
}

lb_status lb_loss_eq6(lb_ctx* c, const void* uref, const void* wref, double Eref, double* loss, void* lam, lb_mem m)
{
    lb_status s = check_ctx(c);
    if (s != LB_OK) return s;
    if (c->stencil != LB_D2Q9) return fail(LB_ERR_UNSUPPORTED, "the Eq. 6 loss is defined for D2Q9");
    if (c->F) return fail(LB_ERR_UNSUPPORTED, "the Eq. 6 loss takes no force");
    if (!uref || !wref || !loss || !mem_valid(m)) return fail(LB_ERR_ARG, "u_ref, w_ref, loss and lb_mem required");
    DeviceGuard guard(c->device);
    Staged su, sw, sl;
    if ((s = stage_in(c, su, uref, 2 * c->N, m, "u_ref")) != LB_OK) return s;
    if ((s = stage_in(c, sw, wref, c->N, m, "w_ref")) != LB_OK) return s;
    if (lam && (s = stage_out_alloc(c, sl, lam, c->N * c->Q, m, false, "lambda")) != LB_OK) return s;
    const int64_t nb = lb::node_grid_blocks(c->g);
    if ((s = ensure_partials(c, 3 * nb + 8)) != LB_OK) return s;
    lb::LossEq6Args e;
    e.a = base_args(c, lb::OP_LOSS_ENERGY);
    e.uref = su.dev;
    e.wref = sw.dev;
    e.Eref = Eref;
    e.lam = lam ? sl.dev : nullptr;
    e.io_f64 = mem_f64(m);
    e.partials = c->partials;
    e.result = c->dsmall;
    e.N = c->N;
    Staged scr;
    scr.c = c;
    if (cudaMallocAsync(&scr.tmp, (size_t)(3 * c->plane * real_bytes(c->opt.storage)), c->stream) != cudaSuccess) {
        scr.tmp = nullptr;
        cudaGetLastError();
        return fail(LB_ERR_OOM, "Eq. 6 scratch");
    }
    e.scratch = scr.tmp;
    int launches = 0;
    cudaError_t ce = lb::loss_eq6_d2q9(e, &launches);
    c->launches += launches;
    if (ce != cudaSuccess) return cuda_fail(c, ce, "Eq. 6 loss");
    LB_CUDA(c, cudaMemcpyAsync(loss, c->dsmall, sizeof(double), cudaMemcpyDeviceToHost, c->stream), "loss read");
    LB_CUDA(c, cudaStreamSynchronize(c->stream), "loss sync");
    if (lam && (s = stage_out_finish(c, sl, lam, "lambda")) != LB_OK) return s;
    return LB_OK;
}

lb_status lb_step_adjoint(lb_ctx* c, const void* lamT, int64_t n, void* lam0, void* gFout, void* gth, lb_mem m)
{
    lb_status s = check_ctx(c);
    if (s != LB_OK) return s;
    if (!lamT || !mem_valid(m)) return fail(LB_ERR_ARG, "lambda_T and a valid lb_mem are required");
    const int k = c->opt.record_every;
    if (k <= 0) return fail(LB_ERR_STATE, "context was created with record_every = 0");
    if (n != c->steps) return fail(LB_ERR_STATE, "n = %lld but %lld steps were recorded", (long long)n, (long long)c->steps);
    if (n > 0 && !c->recording) return fail(LB_ERR_STATE, "no recorded run");
    if (gth && !is_learned(c->coll)) return fail(LB_ERR_ARG, "grad_theta needs a learned collision");
    if (c->coll == LB_TRT || c->coll == LB_KBC || c->coll == LB_MRT)
        return fail(LB_ERR_UNSUPPORTED, "no adjoint of the TRT, KBC or MRT collision");
    if (c->links) return fail(LB_ERR_UNSUPPORTED, "no adjoint with walls");
    DeviceGuard guard(c->device);
    const int f64 = c->opt.storage == LB_F64;
    const int64_t rb = real_pop_bytes(c);
    for (int b = 0; b < 2; ++b)
        if (!c->lam[b] && (s = alloc(c, &c->lam[b], rb, "adjoint buffer")) != LB_OK) return s;
    const int64_t gFb = (int64_t)c->D * c->plane * real_bytes(c->opt.storage);
    if (c->F && !c->gF && (s = alloc(c, &c->gF, gFb, "force gradient")) != LB_OK) return s;
    while ((int64_t)c->ring.size() < k - 1) {
        void* p = nullptr;
        if ((s = alloc(c, &p, pop_bytes(c), "recompute buffer")) != LB_OK) return s;
        c->ring.push_back(p);
    }
    int64_t nblk = 0;
    const int ntheta = net_theta(c->coll);
    if (is_learned(c->coll)) {
        nblk = lb::learned_adj_partial_count(c->g, c->opt.storage, c->sms, c->coll == LB_LEARNED_MRT3);
        const int64_t need = nblk * ntheta;
        // block partials, then the chunk sums of the deterministic reduction
        const int64_t bytes = need * real_bytes(c->opt.storage) + lb::learned_theta_chunk_doubles() * 8 + 256;
        if (c->gtheta_cap < bytes) {
            if (c->gtheta) cudaFree(c->gtheta);
            c->gtheta = nullptr;
            c->gtheta_cap = 0;
            if ((s = alloc(c, &c->gtheta, bytes, "parameter gradient")) != LB_OK) return s;
            c->gtheta_cap = bytes;
        }
        LB_CUDA(c, cudaMemsetAsync(c->gtheta, 0, (size_t)(need * real_bytes(c->opt.storage)), c->stream), "gtheta clear");
    }
    // lambda^n from the caller
    Staged sl;
    if ((s = stage_in(c, sl, lamT, c->N * c->Q, m, "lambda_T")) != LB_OK) return s;
    LB_CUDA(c, lb::convert_copy(sl.dev, mem_f64(m), c->lam[0], f64, c->N, c->N, c->plane, c->Q, 0, c->stream),
            "lambda_T copy");
    c->launches += 1;
    if (c->gF) LB_CUDA(c, cudaMemsetAsync(c->gF, 0, (size_t)gFb, c->stream), "gF clear");
    int cur = 0;
    const int64_t nseg = (n + k - 1) / k;
    std::vector<void*> states((size_t)k);
    for (int64_t seg = nseg - 1; seg >= 0; --seg) {
        const int64_t start = seg * k;
        const int64_t L = (n - start < k) ? n - start : k;
        states[0] = c->ckpt[(size_t)seg];
        for (int64_t j = 1; j < L; ++j) {
            lb::OpArgs a = base_args(c, lb::OP_UPDATE);
            a.mode = lb::AB;
            a.src = states[(size_t)(j - 1)];
            a.dst = c->ring[(size_t)(j - 1)];
            if ((s = launch(c, a, "recompute")) != LB_OK) return s;
            states[(size_t)j] = c->ring[(size_t)(j - 1)];
        }
        for (int64_t j = L - 1; j >= 0; --j) {
            lb::OpArgs a = base_args(c, lb::OP_ADJ_STEP);
            a.mode = lb::AB;
            a.src = states[(size_t)j];
            a.lam_in = c->lam[cur];
            a.lam_out = c->lam[1 - cur];
            a.gF = c->gF;
            a.gth = c->gtheta;
            if ((s = launch(c, a, "adjoint step")) != LB_OK) return s;
            cur = 1 - cur;
        }
    }
    if (lam0) {
        Staged so;
        if ((s = stage_out_alloc(c, so, lam0, c->N * c->Q, m, false, "lambda_0")) != LB_OK) return s;
        LB_CUDA(c, lb::convert_copy(c->lam[cur], f64, so.dev, mem_f64(m), c->N, c->plane, c->N, c->Q, 0, c->stream),
                "lambda_0 copy");
        c->launches += 1;
        if ((s = stage_out_finish(c, so, lam0, "lambda_0")) != LB_OK) return s;
    }
    if (gFout && c->gF) {
        Staged so;
        if ((s = stage_out_alloc(c, so, gFout, c->N * c->D, m, true, "grad_F")) != LB_OK) return s;
        LB_CUDA(c, lb::convert_copy(c->gF, f64, so.dev, mem_f64(m), c->N, c->plane, c->N, c->D, 1, c->stream),
                "grad_F copy");
        c->launches += 1;
        if ((s = stage_out_finish(c, so, gFout, "grad_F")) != LB_OK) return s;
    }
    if (gth) {
        Staged so;
        if ((s = stage_out_alloc(c, so, gth, ntheta, m, true, "grad_theta")) != LB_OK) return s;
        const int64_t part_bytes = nblk * ntheta * real_bytes(c->opt.storage);
        double* chunk = (double*)((char*)c->gtheta + (part_bytes + 255) / 256 * 256);
        LB_CUDA(c, lb::learned_reduce_theta(c->gtheta, nblk, ntheta, f64, chunk, so.dev, mem_f64(m), c->stream),
                "grad_theta");
        c->launches += 2;
        if ((s = stage_out_finish(c, so, gth, "grad_theta")) != LB_OK) return s;
    }
    return LB_OK;
}

lb_status lb_coarsen_into(const lb_ctx* fine_c, lb_ctx* c)
{
    lb_ctx* f = const_cast<lb_ctx*>(fine_c);
    lb_status s = check_ctx(f);
    if (s != LB_OK) return s;
    if ((s = check_ctx(c)) != LB_OK) return s;
    if (f->stencil != c->stencil) return fail(LB_ERR_ARG, "coarsening needs the same velocity set");
    if (f->device != c->device) return fail(LB_ERR_ARG, "coarsening needs both contexts on one device");
    for (int a = 0; a < f->D; ++a)
        if (f->dims[a] != 2 * c->dims[a]) return fail(LB_ERR_ARG, "fine dims must be twice the coarse dims");
    DeviceGuard guard(c->device);
    // work on the fine context's stream, then order the coarse stream after it
    double *rf = nullptr, *uf = nullptr, *rc = nullptr, *uc = nullptr;
    cudaStream_t st = f->stream;
    LB_CUDA(c, cudaMallocAsync((void**)&rf, (size_t)(f->N * 8), st), "coarsen scratch");
    LB_CUDA(c, cudaMallocAsync((void**)&uf, (size_t)(f->N * f->D * 8), st), "coarsen scratch");
    LB_CUDA(c, cudaMallocAsync((void**)&rc, (size_t)(c->N * 8), st), "coarsen scratch");
    LB_CUDA(c, cudaMallocAsync((void**)&uc, (size_t)(c->N * c->D * 8), st), "coarsen scratch");
    lb::OpArgs a = base_args(f, lb::OP_MOMENTS);
    a.out0 = rf;
    a.out1 = uf;
    a.io_f64 = 1;
    if ((s = launch(f, a, "coarsen moments")) != LB_OK) return s;
    LB_CUDA(c, lb::coarsen2(rf, uf, (int)f->dims[0], (int)f->dims[1], (int)f->dims[2], f->D, rc, uc, st), "coarsen");
    f->launches += 1;
    if (c->stream != st) {
        cudaEvent_t ev;
        LB_CUDA(c, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "coarsen event");
        LB_CUDA(c, cudaEventRecord(ev, st), "coarsen event");
        LB_CUDA(c, cudaStreamWaitEvent(c->stream, ev, 0), "coarsen event");
        cudaEventDestroy(ev);
    }
    c->aa_parity = 0;
    c->state = c->ab[0];
    lb::OpArgs b = base_args(c, lb::OP_INIT_EQ);
    b.dst = c->state;
    b.in0 = rc;
    b.in1 = uc;
    b.io_f64 = 1;
    if ((s = launch(c, b, "coarse init")) != LB_OK) return s;
    reset_recording(c);
    if (c->stream != st) LB_CUDA(c, cudaStreamSynchronize(c->stream), "coarsen sync");
    cudaFreeAsync(rf, st);
    cudaFreeAsync(uf, st);
    cudaFreeAsync(rc, st);
    cudaFreeAsync(uc, st);
    return LB_OK;
}

lb_status lb_vorticity(lb_ctx* c, void* w, lb_mem m)
{
    lb_status s = check_ctx(c);
    if (s != LB_OK) return s;
    if (c->stencil != LB_D2Q9) return fail(LB_ERR_UNSUPPORTED, "vorticity is provided for D2Q9");
    if (!w || !mem_valid(m)) return fail(LB_ERR_ARG, "w and a valid lb_mem are required");
    DeviceGuard guard(c->device);
    double* u = nullptr;
    LB_CUDA(c, cudaMallocAsync((void**)&u, (size_t)(c->N * 2 * 8), c->stream), "vorticity scratch");
    lb::OpArgs a = base_args(c, lb::OP_MOMENTS);
    a.out0 = nullptr;
    a.out1 = u;
    a.io_f64 = 1;
    if ((s = launch(c, a, "vorticity moments")) != LB_OK) return s;
    Staged sw;
    if ((s = stage_out_alloc(c, sw, w, c->N, m, false, "vorticity")) != LB_OK) return s;
    LB_CUDA(c, lb::vorticity2d(u, (int)c->dims[0], (int)c->dims[1], sw.dev, mem_f64(m), c->stream), "vorticity");
    c->launches += 1;
    cudaFreeAsync(u, c->stream);
    return stage_out_finish(c, sw, w, "vorticity");
}

lb_status lb_learned_inputs(lb_ctx* c, void* I, lb_mem m)
{
    lb_status s = check_ctx(c);
    if (s != LB_OK) return s;
    if (c->stencil != LB_D2Q9) return fail(LB_ERR_UNSUPPORTED, "the learned collision's inputs are defined for D2Q9");
    if (!I || !mem_valid(m)) return fail(LB_ERR_ARG, "I and a valid lb_mem are required");
    DeviceGuard guard(c->device);
    Staged so;
    if ((s = stage_out_alloc(c, so, I, 6 * c->N, m, false, "inputs")) != LB_OK) return s;
    lb::OpArgs a = base_args(c, lb::OP_MOMENTS);
    a.out0 = so.dev;
    a.io_f64 = mem_f64(m);
    cudaError_t e = lb::learned_inputs_d2q9(a);
    c->launches += 1;
    if (e != cudaSuccess) return cuda_fail(c, e, "learned inputs");
    return stage_out_finish(c, so, I, "inputs");
}

lb_status lb_adam_update(float* theta, float* mm, float* v, const float* g, int64_t n, double lr, double b1, double b2,
                         double eps, int64_t t, void* stream)
{
    if (!theta || !mm || !v || !g || n < 0 || t < 1) return fail(LB_ERR_ARG, "bad Adam arguments");
    const double c1 = 1.0 - std::pow(b1, (double)t), c2 = 1.0 - std::pow(b2, (double)t);
    cudaError_t e = lb::adam_update(theta, mm, v, g, n, (float)lr, (float)b1, (float)b2, (float)eps, (float)c1,
                                    (float)c2, (cudaStream_t)stream);
    if (e != cudaSuccess) return fail(LB_ERR_CUDA, "adam: %s", cudaGetErrorString(e));
    return LB_OK;
}

lb_status lb_stream_copy(const void* src, void* dst, int64_t bytes, void* stream)
{
    if (!src || !dst) return fail(LB_ERR_ARG, "lb_stream_copy: null pointer");
    if (bytes <= 0 || bytes % 16 != 0) return fail(LB_ERR_ARG, "lb_stream_copy: bytes must be a positive multiple of 16");
    if (((uintptr_t)src | (uintptr_t)dst) % 16 != 0)
        return fail(LB_ERR_ARG, "lb_stream_copy: pointers must be 16-byte aligned");
    int cur = -1, sms = 0;
    if (cudaGetDevice(&cur) != cudaSuccess) return fail(LB_ERR_CUDA, "lb_stream_copy: no current device");
    for (const void* p : {src, (const void*)dst}) {
        cudaPointerAttributes attr;
        if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
            cudaGetLastError();  // clear the (non-sticky) error the failed query recorded
            return fail(LB_ERR_ARG, "lb_stream_copy: not a CUDA pointer");
        }
        if (!((attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged) && attr.device == cur))
            return fail(LB_ERR_ARG, "lb_stream_copy: src and dst must be device (or managed) memory of the current device");
    }
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, cur) != cudaSuccess)
        return fail(LB_ERR_CUDA, "lb_stream_copy: device query failed");
    const cudaError_t e = lb::stream_copy(src, dst, bytes, sms, (cudaStream_t)stream);
    if (e != cudaSuccess) return fail(LB_ERR_CUDA, "lb_stream_copy: %s", cudaGetErrorString(e));
    return LB_OK;
}

int64_t lb_num_nodes(const lb_ctx* c) { return c ? c->N : -1; }
int lb_q(const lb_ctx* c) { return c ? c->Q : -1; }
int lb_d(const lb_ctx* c) { return c ? c->D : -1; }
int64_t lb_launch_count(const lb_ctx* c) { return c ? c->launches : -1; }

const char* lb_status_string(lb_status s)
{
    switch (s) {
    case LB_OK: return "ok";
    case LB_ERR_ARG: return "invalid argument";
    case LB_ERR_OOM: return "out of device memory";
    case LB_ERR_CUDA: return "CUDA error";
    case LB_ERR_UNSTABLE: return "unstable (non-finite or non-positive density)";
    case LB_ERR_STATE: return "invalid state";
    case LB_ERR_UNSUPPORTED: return "unsupported";
    default: return "unknown status";
    }
}

const char* lb_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
