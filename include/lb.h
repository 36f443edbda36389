/*
 * liblb — lattice Boltzmann stream-and-collide on one GB300 (sm_103a), C ABI.
 *
 * The library advances the particle populations f_i(x, t) of a periodic Cartesian
 * grid by the lattice Boltzmann equation f_i(x + c_i, t + 1) = f_i(x, t) + Omega_i(f)
 * (Bedrunka et al., arXiv 2106.12929, Sec. 2.1, Eq. 1) with
 *   - the D2Q9, D3Q19 and D3Q27 velocity sets (Sec. 2.2, 3.1, 3.3),
 *   - the second-order equilibrium (Eq. 3) and the moments rho, rho u (Eq. 4),
 *   - BGK (Eq. 2), regularized (Sec. 2.1) or moment-space collision with learned
 *     higher-moment relaxation rates (Eq. 5, Sec. 3.1: a shared rate from a 6-24-24-1
 *     network, or three rates from the paper's one-hidden-layer network), the further
 *     models Sec. 2.1 cites (TRT, entropic KBC, MRT with fixed rates), and a Guo body force,
 *   - halfway bounce-back walls on solid nodes (Sec. 2.2 lists boundary conditions),
 * plus the discrete adjoint of the time stepping (gradients through the solver,
 * Sec. 3.2), the Eq. 6 training loss and its training helpers, and the spectral flow
 * control of Sec. 3.2 (every step a velocity shift down the gradient of a log-spectrum
 * mismatch).
 *
 * Conventions for every call
 *   - Grid: dims = {nx, ny, nz}; 2D stencils need nz == 1. Node n = x + nx (y + ny z).
 *     N = nx ny nz nodes, 1 <= nx, ny, nz <= 65535 and N < 2^31 (LB_ERR_ARG otherwise).
 *     Every direction is periodic (walls are solid
 *     nodes set by lb_set_solid).
 *   - Arrays crossing the boundary are dense, component-major, x fastest:
 *     populations f[Q][N], velocity u[d][N], force F[d][N], density rho[N].
 *     Their element type and location are given by an lb_mem value; device pointers
 *     must be on the context's device. The caller owns every buffer it passes; the
 *     library copies in or out on the context's stream and keeps no pointer to it.
 *   - The exposed state is always the PRE-collision state f^n of Eq. 1, whatever
 *     the internal layout (two-buffer pull, or in-place AA) and storage type.
 *   - Calls are asynchronous on the context's stream except where a result is
 *     returned in host memory (those synchronise the stream before returning).
 *   - Errors are returned as lb_status; nothing aborts, exits or traps. On an
 *     argument error the context is unchanged. On a CUDA error the context is
 *     marked failed and every later call returns LB_ERR_STATE. lb_last_error()
 *     gives a message for the calling thread.
 *   - A context is not thread safe; use one context per thread or lock around it.
 */
#ifndef LIBLB_LB_H
#define LIBLB_LB_H

#include <stdint.h>

#if defined(__GNUC__)
#define LB_API __attribute__((visibility("default")))
#else
#define LB_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lb_ctx lb_ctx; /* opaque, owned by the library */

typedef enum { LB_D2Q9 = 0, LB_D3Q19 = 1, LB_D3Q27 = 2 } lb_stencil;

/* Collision operator.
 *   LB_BGK          Eq. 2: f* = f - (f - f^eq)/tau (+ Guo source).
 *   LB_REGULARIZED  Latt & Chopard (Sec. 2.1): relax only the projection of f - f^eq
 *                   onto the Hermite polynomials of order <= 2 (+ Guo source).
 *   LB_LEARNED_MRT  Eq. 5 on D2Q9: Hermite moments; stress rows relax with 1/tau,
 *                   the three higher rows with 1/(exp(z) + 1/2), z = a per-node
 *                   6-24-24-1 tanh network of local moment invariants (Sec. 3.1).
 *                   No body force.
 *   LB_NONE         streaming only (f* = f); the force is ignored. For tests.
 * Further models the paper lists by citation (Sec. 2.1); no adjoint, no recording:
 *   LB_TRT          two relaxation times (Ginzburg): the symmetric half of f - f^eq of
 *                   each pair (i, opposite i) relaxes with 1/tau, the antisymmetric half
 *                   with 1/tau_minus, tau_minus = 1/2 + Lambda/(tau - 1/2); Lambda = 1/4
 *                   unless set by lb_set_relaxation. Guo source split the same way. Any set.
 *   LB_KBC          entropic KBC (Karlin, Boesch & Chikatamarla): f - f^eq = Ds + Dh with
 *                   Ds the trace-free second natural moments; f* = f - beta (2 Ds + gamma Dh),
 *                   beta = 1/(2 tau), gamma = 1/beta - (2 - 1/beta) <Ds|Dh> / (<Dh|Dh> +
 *                   1e-6 <Ds|Ds>), <X|Y> = sum X_i Y_i / f^eq_i. D2Q9 and D3Q27; no force.
 *   LB_MRT          Eq. 5 with fixed rates on D2Q9: stress moments relax with 1/tau, the
 *                   three higher Hermite moments with 1/tau_6, 1/tau_7, 1/tau_8 (1 unless
 *                   set by lb_set_relaxation). No force.
 *   LB_LEARNED_MRT3 Eq. 5 on D2Q9 with the network shape Sec. 3.1 describes: one hidden
 *                   layer of 53 tanh units and three outputs z_0, z_1, z_2, each giving one
 *                   higher moment its own relaxation time exp(z) + 1/2, in the order the
 *                   paper lists those moments: the fourth-order moment
 *                   (cx^2 - 1/3)(cy^2 - 1/3), then the third-order (cx^2 - 1/3) cy and
 *                   cx (cy^2 - 1/3). Same inputs as LB_LEARNED_MRT; 533 trained
 *                   parameters. With adjoint and parameter gradient. No force. */
typedef enum {
    LB_BGK = 0,
    LB_REGULARIZED = 1,
    LB_LEARNED_MRT = 2,
    LB_NONE = 3,
    LB_TRT = 4,
    LB_KBC = 5,
    LB_MRT = 6,
    LB_LEARNED_MRT3 = 7
} lb_collision;

/* Storage of the populations in device memory. Arithmetic is FP64 for LB_F64 and
 * FP32 otherwise. LB_F32 and the half types store the shifted value f_i - w_i (the
 * deviation from rest, 10 to 40 times smaller than f_i near rest, so its rounding is that
 * much smaller), rounded to nearest even; LB_F64 stores f_i. Every accessor exposes f_i. */
typedef enum { LB_F64 = 0, LB_F32 = 1, LB_F16_SHIFTED = 2, LB_BF16_SHIFTED = 3 } lb_storage;

/* LB_LAYOUT_AB: two population buffers, one fused pull-stream + collide launch per
 *               step from one into the other.
 * LB_LAYOUT_AA: one buffer updated in place, alternating even and odd steps
 *               (half the memory of AB, the same bytes moved per step). */
typedef enum { LB_LAYOUT_AB = 0, LB_LAYOUT_AA = 1 } lb_layout;

/* Element type and location of an array argument. A host array in page-locked memory (pinned
 * or registered with CUDA) is read, or written, in place by the call's kernels through its
 * device address (over NVLink-C2C on Grace-Blackwell); a pageable host array, and an output
 * that a call accumulates into (grad_F, grad_theta), go through a stream-ordered temporary
 * device buffer and a copy. Either way a call returns its host outputs complete; host inputs
 * must stay unchanged until the stream has run the call's work. */
typedef enum { LB_HOST_F64 = 0, LB_DEVICE_F64 = 1, LB_HOST_F32 = 2, LB_DEVICE_F32 = 3 } lb_mem;

typedef enum {
    LB_OK = 0,
    LB_ERR_ARG = 1,         /* bad argument; nothing was done */
    LB_ERR_OOM = 2,         /* device allocation failed */
    LB_ERR_CUDA = 3,        /* a CUDA call failed; the context is now failed */
    LB_ERR_UNSTABLE = 4,    /* a node had a non-finite or non-positive density */
    LB_ERR_STATE = 5,       /* call not valid in the current state (or context failed) */
    LB_ERR_UNSUPPORTED = 6  /* valid but not provided (e.g. learned collision on D3Q19) */
} lb_status;

typedef struct {
    lb_storage storage;   /* default LB_F32 */
    lb_layout layout;     /* default LB_LAYOUT_AB */
    void* cuda_stream;    /* cudaStream_t of all work; NULL = the legacy default stream */
    int device;           /* CUDA device ordinal; -1 (default) = the current device */
    int check_every;      /* >0: lb_step synchronises every check_every steps and at its end
                             and returns LB_ERR_UNSTABLE if a node went bad; 0 (default) = never */
    int record_every;     /* >0: lb_step records a checkpoint every record_every steps so that
                             lb_step_adjoint can run backwards (AB layout only); 0 = off */
    int learned_tc;       /* LB_LEARNED_MRT(3), FP32/FP16/BF16 storage: 1 = evaluate the network in
                             half precision (FP16 operands, FP16 accumulation in the hidden layers,
                             the hardware tanh; an inference option: lb_step_adjoint and training
                             use the default path; grids up to about 238 million nodes, 9 x the
                             padded plane below 2^31); 0 (default) = the FP32 network: its matrix products on the tensor cores,
                             each operand split into two FP16 terms and multiplied as
                             hi.hi + hi.lo + lo.hi (about 2^-21 relative; operands scaled by
                             powers of two into FP16 range), an FP32 tanh, FP32 everything else */
    int graphs;           /* 1 (default): lb_step(n >= 2) without checkpoints captures two steps once
                             into a CUDA graph and replays it (one launch per pair of steps instead
                             of one per kernel; same kernels, same results); 0 = direct launches */
    int nodes_per_thread; /* shape of the stream-collide launch: 0 (default) = chosen from the grid
                             (one node per thread in 32-thread blocks when the grid has fewer
                             256-node x-rows than SMs, else four per thread for half storage
                             without a force (except D3Q27 KBC), two otherwise);
                             1, 2 or 4 = forced, falling back to the next smaller shape the grid
                             allows (2 needs an even nx; 4 needs half storage and nx % 4 == 0).
                             LB_NONE and the learned collisions always run one node per thread.
                             The shapes agree to the last bits of the arithmetic type (the
                             compiler contracts multiply-adds differently per shape); one
                             shape always gives the same bits */
} lb_options;

/* Fill *opt with the defaults listed above (learned_tc = 0, graphs = 1, nodes_per_thread = 0). */
LB_API void lb_default_options(lb_options* opt);

/* Create a context: validate, allocate the population buffer(s) on opt->device and
 * zero them. tau > 1/2 is the BGK relaxation time of Eq. 2 (viscosity
 * nu = c_s^2 (tau - 1/2)); for LB_LEARNED_MRT it is the stress relaxation time
 * tau_n of Sec. 3.1. opt may be NULL (defaults). On success *out owns the memory
 * until lb_destroy. Errors: LB_ERR_ARG (dims, tau, enum values, option values),
 * LB_ERR_UNSUPPORTED (the learned collisions or MRT on a stencil other than D2Q9, KBC on
 * D3Q19, learned_tc without a learned collision, with FP64 storage or on a grid whose
 * 9 x padded plane reaches 2^31, record_every with the AA layout or with TRT, KBC or MRT),
 * LB_ERR_OOM, LB_ERR_CUDA. */
LB_API lb_status lb_create(lb_ctx** out, lb_stencil stencil, const int64_t dims[3], double tau,
                    lb_collision collision, const lb_options* opt);

/* Release every device buffer of the context (synchronises its stream). NULL is a no-op. */
LB_API void lb_destroy(lb_ctx* ctx);

/* f_i = f_i^eq(rho, u) at every node (Eq. 3), as the pre-collision state f^0.
 * rho[N], u[d][N]. The velocity is used as given (no force shift). Resets the
 * step counter and any recording. */
LB_API lb_status lb_init_from_moments(lb_ctx* ctx, const void* rho, const void* u, lb_mem mem);

/* Set the body force F[d][N] (constant in time); NULL clears it. The velocity of a
 * forced state is u = (sum_i c_i f_i + F/2)/rho and the Guo source
 * S_i = (1 - omega/2) w_i [(c_i - u)/c_s^2 + (c_i . u) c_i / c_s^4] . F is added in
 * the collision (Guo, Zheng & Shi 2002; the paper only mentions forcing, Sec. 2.2).
 * LB_ERR_UNSUPPORTED with the learned, KBC or MRT collisions or with the spectral
 * control on. */
LB_API lb_status lb_set_force(lb_ctx* ctx, const void* F, lb_mem mem);

/* Network of the learned collision (Sec. 3.1).
 * LB_LEARNED_MRT, n_params = 805 values: W1[24][6], b1[24], W2[24][24], b2[24], W3[24],
 * b3 (793 trained parameters), then the fixed input shift[6] and scale[6] (input k is
 * (I_k - shift_k) scale_k).
 * LB_LEARNED_MRT3, n_params = 545 values: W1[53][6], b1[53], W2[3][53], b2[3] (533 trained
 * parameters; output 0 sets the fourth-order moment's time, outputs 1 and 2 the
 * third-order ones, see lb_collision), then shift[6] and scale[6] as above.
 * LB_ERR_STATE for other collisions, LB_ERR_ARG for another count or a non-finite value. */
LB_API lb_status lb_set_mlp(lb_ctx* ctx, const void* params, int64_t n_params, lb_mem mem);

/* Further relaxation parameters (host memory, copied): LB_TRT n = 1, params[0] =
 * Lambda = (tau - 1/2)(tau_minus - 1/2) > 0 (1/4 by default; (tau - 1/2)^2 gives BGK);
 * LB_MRT n = 3, params = tau_6, tau_7, tau_8 > 1/2, the relaxation times of the higher
 * moments (cx^2 - 1/3) cy, cx (cy^2 - 1/3), (cx^2 - 1/3)(cy^2 - 1/3) (1, 1, 1 by default;
 * all equal to tau gives BGK). LB_ERR_STATE for other collisions, LB_ERR_ARG for a
 * wrong count or value. Applies from the next lb_step. */
LB_API lb_status lb_set_relaxation(lb_ctx* ctx, const double* params, int n);

/* Solid nodes with halfway bounce-back (the paper lists boundary conditions without
 * formulas, Sec. 2.2; textbook form with Ladd's moving-wall term). mask: N bytes in x-fastest
 * node order, nonzero = solid, on the host or the device as mem says (the element type of
 * mem applies to wall_u only). A fluid node's population that would stream into a solid
 * node returns to it in the opposite direction at the next step:
 *   f_opp(i)(x, t + 1) = f*_i(x, t) - 2 w_i (c_i . u_w) / c_s^2,
 * u_w = wall_u at the solid node x + c_i (wall density 1; wall_u [d][N] or NULL = resting
 * walls). Solid nodes do not collide; their exposed state is the rest equilibrium f_i = w_i.
 * mask NULL removes all walls. AB layout only, not with the learned collisions, recording
 * or the spectral control (LB_ERR_UNSUPPORTED). Copies both arrays. */
LB_API lb_status lb_set_solid(lb_ctx* ctx, const void* mask, const void* wall_u, lb_mem mem);

/* Advance n >= 0 steps of Eq. 1: one fused kernel launch per step (five with the spectral
 * control on); with graphs on and no recording, pairs of steps replay one captured CUDA
 * graph. With check_every > 0 returns LB_ERR_UNSTABLE as described in lb_options. */
LB_API lb_status lb_step(lb_ctx* ctx, int64_t n);

/* rho[N] and u[d][N] of the current pre-collision state (Eq. 4, with the force
 * shift if a force is set). Either pointer may be NULL. */
LB_API lb_status lb_moments(lb_ctx* ctx, void* rho, void* u, lb_mem mem);

/* Global sums of the current state, accumulated in FP64 in a fixed order
 * (deterministic): the mass and momentum that the collision conserves (Sec. 2.1) and the
 * kinetic energy the paper reports as its observable (Sec. 2.2, the energy of the Taylor-Green
 * vortex): out[0] = sum rho, out[1..3] = sum rho u (x, y, z; z = 0 in 2D),
 * out[4] = (1/2N) sum |u|^2 (incompressible kinetic energy), out[5] = (1/2N) sum rho |u|^2.
 * out is host memory; the call synchronises the stream. */
LB_API lb_status lb_reduce(lb_ctx* ctx, double out[6]);

/* Copy the current pre-collision state f^n of Eq. 1 out as f[Q][N] (natural layout,
 * unshifted), e.g. for a checkpoint; the paper has no counterpart for the copy itself. */
LB_API lb_status lb_get_populations(lb_ctx* ctx, void* f, lb_mem mem);

/* Replace the state by f[Q][N], taken as the pre-collision f^n of Eq. 1 (natural layout;
 * a checkpoint's restart or an arbitrary initial state, where lb_init_from_moments gives only
 * equilibria). Resets the step counter and any recording. */
LB_API lb_status lb_set_populations(lb_ctx* ctx, const void* f, lb_mem mem);

/* Synchronise the stream and report LB_ERR_UNSTABLE if any node of any step since
 * the last check had a non-finite or non-positive density (the flag is then cleared).
 * Failure detection of this library; the paper has no counterpart (a BGK run that leaves its
 * stability range, Sec. 3.1, shows up here). */
LB_API lb_status lb_check(lb_ctx* ctx);

/* Steps taken since the last initialisation. */
LB_API int64_t lb_steps_taken(const lb_ctx* ctx);

/* ----------------------------------------------------- spectral flow control ---- */
/* Sec. 3.2 keeps a flow's energy spectrum near a target sigma_0 by a velocity-shift
 * forcing: every step collides with BGK (Eq. 2) at the equilibrium f^eq(rho, u + du),
 * du = -kappa grad_u R, where
 *   R(u) = sum_s (ln max(sigma_s(u), c) - ln max(sigma0_s, c))^2
 * and sigma_s(u) = sum over the Fourier modes k with round(|k|) = s of
 * (|u_hat_x(k)|^2 + |u_hat_y(k)|^2) / 2, u_hat = (1/N) sum_x u(x) exp(-2 pi i k.x / n), for
 * the shells s = 0 .. n/2 - 1 (the paper does not define the spectrum's normalisation or
 * shells; this is its reading). The paper's constants are c = 2e-5 and kappa = 5e-5.
 * grad_u R is the exact gradient of R (a spectral filter of u), computed each step on the
 * GPU by FFTs of the grid lines. D2Q9 only, on a square grid of n = 2^k nodes per side,
 * 4 <= n <= 4096, any storage and layout. The first spectral call on a context allocates its
 * scratch, kept until lb_destroy: the complex field (n^2 values of the arithmetic type), the
 * line transforms' tables (the twiddles, the shell of every mode as int16, the first |ky| of
 * every shell per column as int16: about 2.5 n^2 bytes), the shell sums and, with the control
 * on, du[2][N]. */

/* Turn the control on (sigma0[K] in host memory, K = n/2 shells, copied; cutoff c > 0,
 * kappa >= 0) or off (sigma0 NULL). From the next lb_step every step computes du from the
 * current state and collides at u + du (five kernel launches per step instead of one).
 * Needs the BGK collision, no force, no walls and record_every = 0 (LB_ERR_UNSUPPORTED
 * otherwise); LB_ERR_ARG for another K or non-finite values. */
LB_API lb_status lb_set_spectral_control(lb_ctx* ctx, const double* sigma0, int64_t K, double cutoff,
                                         double kappa);

/* Spectrum sigma[n/2] of the current state (host memory, FP64; may be NULL) and, when the
 * control is on, its cost R (*cost, host; may be NULL; LB_ERR_STATE without a target).
 * Square 2^k D2Q9 grids only (LB_ERR_UNSUPPORTED). Synchronises the stream. */
LB_API lb_status lb_spectrum(lb_ctx* ctx, double* sigma, double* cost);

/* The velocity shift du[2][N] = -kappa grad_u R of the current state, as the next step
 * would apply it (control on, else LB_ERR_STATE). */
LB_API lb_status lb_spectral_shift(lb_ctx* ctx, void* du, lb_mem mem);

/* ------------------------------------------------------------------ adjoint ---- */
/* The discrete adjoint of f^{n+1} = S C(f^n; F), S the periodic shift along c_i
 * (Sec. 3.2 takes such gradients by automatic differentiation; here they are
 * written out): lambda^n = J_C(f^n; F)^T S^T lambda^{n+1}, dL/dF += (dC/dF)^T S^T lambda^{n+1}. */

/* Seed from moment cotangents of the current state: given dL/drho[N] (may be NULL)
 * and dL/du[d][N], write lambda = dL/df [Q][N] and add the force's direct part
 * dL/du / (2 rho) to grad_F[d][N] (grad_F may be NULL). */
LB_API lb_status lb_adjoint_seed_moments(lb_ctx* ctx, const void* grad_rho, const void* grad_u, void* lambda,
                                  void* grad_F, lb_mem mem);

/* Kinetic-energy-field loss L = sum_x (e(x) - e*(x))^2, e = rho |u|^2 / 2, of the
 * current state: *loss (host, FP64), lambda = dL/df [Q][N], grad_F += dL/dF's direct
 * part (may be NULL). e_target[N]. Synchronises the stream. */
LB_API lb_status lb_loss_energy(lb_ctx* ctx, const void* e_target, double* loss, void* lambda, void* grad_F,
                         lb_mem mem);

/* Eq. 6 loss of the current D2Q9 state against targets u_ref[2][N], w_ref[N] (vorticity)
 * and E_ref: L = 0.6 mean|u - u_ref|^2 + 0.2 mean(w - w_ref)^2 + 0.2 (E - E_ref)^2 with
 * w by central differences and E = (1/2N) sum |u|^2. *loss (host, FP64) and
 * lambda = dL/df [Q][N]. No force. Synchronises the stream. */
LB_API lb_status lb_loss_eq6(lb_ctx* ctx, const void* u_ref, const void* w_ref, double E_ref, double* loss,
                      void* lambda, lb_mem mem);

/* Run the adjoint back over the n steps recorded since the last initialisation
 * (n must equal lb_steps_taken and the context must have record_every > 0).
 * lambda_T[Q][N] = dL/df^n of the current state. Outputs (each may be NULL):
 * lambda_0[Q][N] = dL/df^0; grad_F[d][N] += dL/dF; grad_theta += dL/dtheta over the
 * trained parameters in lb_set_mlp's order (learned collisions only: 793 values for
 * LB_LEARNED_MRT, 533 for LB_LEARNED_MRT3). Recomputes each checkpoint segment forward once.
 * The state is left at f^n. */
LB_API lb_status lb_step_adjoint(lb_ctx* ctx, const void* lambda_T, int64_t n, void* lambda_0, void* grad_F,
                          void* grad_theta, lb_mem mem);

/* The six inputs of the learned collision's network at every node of the current
 * D2Q9 state, before standardisation (Sec. 3.1 "local moments"; see lb_set_mlp):
 * I[0] = rho - 1, I[1] = |u|^2/c_s^2, I[2] = tr Pi/c_s^2, I[3] = Pi:Pi/c_s^4,
 * I[4] = u.Pi.u/c_s^4, I[5] = sum of the squared higher (ghost) moments over their
 * weighted norms; Pi = sum c c (f - f^eq). Layout I[6][N]. Any collision kind. */
LB_API lb_status lb_learned_inputs(lb_ctx* ctx, void* I, lb_mem mem);

/* Coarse-graining used to build training data (Sec. 3.1: the fine trajectory is
 * mapped onto a grid with half the resolution): the coarse context's state becomes
 * f^eq(rho_c, u_c), where rho_c and rho_c u_c are the means of rho and rho u over each
 * 2 x 2 (x 2) block of the fine context's current state. Same velocity set, fine
 * dims = 2 x coarse dims, one device. Resets the coarse step counter and recording. */
LB_API lb_status lb_coarsen_into(const lb_ctx* fine, lb_ctx* coarse);

/* Vorticity w[N] = (v(x+1) - v(x-1))/2 - (u(y+1) - u(y-1))/2 of the current D2Q9 state
 * (the Eq. 6 vorticity, second-order central differences on the periodic grid). */
LB_API lb_status lb_vorticity(lb_ctx* ctx, void* w, lb_mem mem);

/* One Adam update of n parameters in device memory (FP32):
 * m = b1 m + (1 - b1) g; v = b2 v + (1 - b2) g^2;
 * theta -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps). t >= 1 is the step
 * number. Runs on `stream` (NULL = legacy default stream). */
LB_API lb_status lb_adam_update(float* theta, float* m, float* v, const float* grad, int64_t n, double lr, double b1,
                         double b2, double eps, int64_t t, void* stream);

/* ------------------------------------------------------------------ slabs ---- */
/* Partitioning across GPUs (the paper names multi-GPU runs as future work, Sec. 3.3): a
 * periodic grid is split along its last axis (z in 3D, y in 2D) into slabs, one per rank.
 * Each rank's context holds its slab plus one ghost layer at each end: its last dimension is
 * the slab's layers + 2, local layer 0 is the ghost below, layer n_last - 1 the ghost above,
 * and the context steps all layers as an ordinary periodic grid (the ghost layers' own
 * updates are discarded). Between steps the populations that cross each face move: the slots
 * whose velocity has last component -1 of interior layer 1 go to the lower neighbour's upper
 * ghost layer, those with +1 of layer n_last - 2 to the upper neighbour's lower ghost layer
 * (3 slots for D2Q9, 5 for D3Q19, 9 for D3Q27). Over an exchanged slab, the interior layers
 * evolve exactly as the same layers of the whole grid with the same launch shape.
 *
 * lb_halo_bytes: size of one face's buffer: crossing slots x layer nodes x the storage's
 * element size (the stored values are copied as they are).
 * lb_halo_pack: copy the crossing populations leaving through `face` (0: low end, 1: high end)
 * into buf; lb_halo_unpack: copy a neighbour's packed buffer into the ghost layer of `face`.
 * buf is device memory of the context's device, laid out [slot][layer nodes]; both calls are
 * ordered on the context's stream and return without synchronising. AB layout only
 * (LB_ERR_UNSUPPORTED otherwise, and for unpacking into a context that records for the
 * adjoint); the last dimension must be >= 3 (LB_ERR_ARG). */
LB_API lb_status lb_halo_bytes(const lb_ctx* ctx, int64_t* bytes);
LB_API lb_status lb_halo_pack(lb_ctx* ctx, int face, void* buf);
LB_API lb_status lb_halo_unpack(lb_ctx* ctx, int face, const void* buf);

/* The global sums of lb_reduce over the layers [first, first + count) of the last axis (a
 * slab's interior: first = 1, count = n_last - 2), unnormalised: out[0] = sum rho,
 * out[1..3] = sum rho u, out[4] = sum |u|^2, out[5] = sum rho |u|^2 (the caller adds the ranks'
 * sums and divides out[4], out[5] by 2 N of the whole grid). FP64, deterministic; out is host
 * memory and the call synchronises the stream. */
LB_API lb_status lb_reduce_slab(lb_ctx* ctx, int64_t first, int64_t count, double out[6]);

/* ------------------------------------------------------- without allocation ---- */
/* The paper has no counterpart to this call; it exists for callers that cannot
 * allocate device memory where they need the global sums: for instance code that
 * has given all device memory to another framework's caching allocator, or a
 * latency-critical loop in which cudaMalloc / cudaFree (which may synchronise the
 * whole device) are not acceptable.
 *
 * Same sums as lb_reduce (out[0] = sum rho, out[1..3] = sum rho u, out[4] =
 * (1/2N) sum |u|^2, out[5] = (1/2N) sum rho |u|^2, FP64, deterministic), but for a
 * caller-owned pre-collision state f[Q][N] in natural layout on the current device,
 * with an optional force F[d][N] (NULL = none) of the same type; mem must be
 * LB_DEVICE_F64 or LB_DEVICE_F32. out is host memory. The work runs on cuda_stream
 * (NULL = legacy default stream) and the call synchronises that stream.
 *
 * It needs no context and performs no device allocation: its per-block partial sums
 * live in a fixed file-scope device array of the library (about 385 KB, held on every
 * GPU that loads the library until the process exits), which limits the grid to
 * N <= 33,554,432 nodes; larger grids are rejected with LB_ERR_ARG. f and F must be
 * device (or managed) memory of the current device (checked with
 * cudaPointerGetAttributes; anything else is LB_ERR_ARG, before any launch). The first
 * call on a device looks up that array's device address (with that device current)
 * and keeps it for the life of the process (do not call this entry point on a device after
 * a cudaDeviceReset). The call synchronises its stream and copies the sums to the host, so it
 * cannot be captured into a CUDA graph. All calls share the array: calls that
 * overlap on the GPU (other streams or threads on the same device) race, so order
 * them. Errors: LB_ERR_ARG (arguments, size), LB_ERR_CUDA. */
LB_API lb_status lb_reduce_noalloc(lb_stencil stencil, const int64_t dims[3], const void* f, const void* F,
                                   lb_mem mem, double out[6], void* cuda_stream);

/* Bandwidth reference for roofline fractions (the paper has no counterpart): copies `bytes`
 * (a positive multiple of 16) from src to dst, both 16-byte aligned device (or managed)
 * memory of the current device holding at least `bytes` (the caller's buffers, not checked
 * beyond their start), as 16-byte vector loads and stores on cuda_stream (NULL = the legacy
 * default stream). Asynchronous: returns after the launch. Errors: LB_ERR_ARG (pointers,
 * alignment, size; before any launch), LB_ERR_CUDA. */
LB_API lb_status lb_stream_copy(const void* src, void* dst, int64_t bytes, void* cuda_stream);

/* ------------------------------------------------------------------ info ---- */
LB_API int64_t lb_num_nodes(const lb_ctx* ctx);
LB_API int lb_q(const lb_ctx* ctx);
LB_API int lb_d(const lb_ctx* ctx);
/* Kernel launches issued by this context since creation (for launch accounting). */
LB_API int64_t lb_launch_count(const lb_ctx* ctx);
LB_API const char* lb_status_string(lb_status s);
/* Message of the last error on the calling thread ("" if none). */
LB_API const char* lb_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* LIBLB_LB_H */
