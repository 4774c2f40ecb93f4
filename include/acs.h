/*
 * acs.h -- C ABI of a GB300 (sm_103a) stepper for the d-dimensional Allen-Cahn
 * equation  phi_t = eps^2 lap(phi) - f(phi),  f(phi) = phi^3 - phi  (d = 1, 2, 3),
 * discretized by the RLB-MIE-FD scheme of Chen, Liu, Chai and Shi,
 * "Regularized lattice Boltzmann method based maximum principle and energy
 * stability preserving finite-difference scheme for the Allen-Cahn equation"
 * (arXiv:2312.07010).
 *
 * One step (Eq. IE-FD, Remark 1), per unknown i:
 *   xi_i  = phi_i + lambda sum_k (phi_{i+e_k} + phi_{i-e_k} - 2 phi_i) - (dt/2) f(phi_i),
 *   phi_i <- the unique real theta with theta + (dt/2) f(theta) = xi_i,
 * with lambda = eps^2 dt / h^2 (Eq. IE-FD-vector-form).  Neighbours outside the
 * box follow the boundary condition (Eq. Ddeltax): periodic = wrap around,
 * Neumann = the node itself (mirror), Dirichlet = 0.
 *
 * Memory layout.  The state is n[0] x ... x n[dims-1] values of the chosen
 * dtype, row-major with the last index fastest (the ordering of Phi in Eq.
 * IE-FD-vector-form), contiguous, in device memory owned by the caller.
 *
 * Ownership.  The library allocates no device memory on these paths: the caller
 * passes the state buffer and a work buffer of acs_work_bytes() bytes (the second
 * ping-pong state plus reduction scratch), and keeps both alive until
 * acs_destroy().  The library owns only the opaque context (host memory), a
 * private CUDA stream used to record CUDA graphs, and those graphs.
 *
 * Streams.  Every device-side call is enqueued on the stream given to acs_bind()
 * and returns without waiting, except the calls that return host values
 * (acs_energy, acs_maxnorm, acs_run_logged, acs_grad, acs_get_state_host,
 * acs_sync), which synchronize that stream.
 *
 * Status codes.  0 = success; > 0 = a warning, the call did its work; < 0 = an
 * error, the call changed nothing that the caller can observe (except where a
 * function says otherwise).  acs_strerror() names each code.
 *
 * Threading.  A context may be used by one host thread at a time.
 */
#ifndef ACS_H
#define ACS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define ACS_API __attribute__((visibility("default")))
#else
#define ACS_API
#endif

typedef struct acs_ctx acs_ctx;
typedef struct acs_batch acs_batch;
typedef struct acs_lines acs_lines;
typedef struct acs_pipe acs_pipe;

/* Boundary conditions (Sec. I: HN-BC, HD-BC, P-BC; matrices of Eq. Ddeltax). */
enum { ACS_BC_PERIODIC = 0, ACS_BC_NEUMANN = 1, ACS_BC_DIRICHLET = 2 };

/* State precision: FP32 state and arithmetic, or FP64.  The energy reduction forms
 * every term of an FP32 state exactly (float pairs from error-free transformations)
 * and sums them in FP64 per thread; FP64 states sum plain FP64 terms per thread (fma,
 * no compensation).  Partial sums of threads and blocks are combined exactly (128-bit
 * fixed point), so the result is deterministic.  The maximum norm is exact. */
enum { ACS_F32 = 0, ACS_F64 = 1 };

/* Status codes. */
enum {
    ACS_OK = 0,
    ACS_WARN_MP_CONDITION = 1,     /* dt > 1 - 2 d lambda: Theorem 2 does not apply */
    ACS_WARN_ENERGY_CONDITION = 2, /* dt > 4 (1 - 2 d lambda): Theorem 3 does not apply */
    ACS_E_INVAL = -1,              /* invalid argument */
    ACS_E_CUDA = -2,               /* a CUDA runtime call failed */
    ACS_E_NOMEM = -3,              /* work buffer too small / host allocation failed */
    ACS_E_TIMEOUT = -4,            /* a bounded device-side wait gave up */
    ACS_E_NONFINITE = -5,          /* the state holds NaN or Inf */
    ACS_E_STATE = -6,              /* call out of order (e.g. step before bind) */
    ACS_E_UNSUPPORTED = -7         /* kernel variant not available for this problem */
};

/* Kernel variants (acs_set_kernel).  The finite-difference variants (1..3) compute
 * the same per-point arithmetic in the same order, so they give bit-identical
 * states.  ACS_KERNEL_LB runs the collide-and-stream form the scheme is derived
 * from (Sec. II): equal to Eq. (IE-FD) up to rounding. */
enum {
    ACS_KERNEL_AUTO = 0,     /* autotuned choice, cached per problem class */
    ACS_KERNEL_NAIVE = 1,    /* one thread per unknown, neighbours via the cache hierarchy */
    ACS_KERNEL_TILED = 2,    /* shared-memory tiles (TMA-staged for d >= 2) with a one-cell halo */
    ACS_KERNEL_TEMPORAL = 3, /* several fused steps per pass through HBM (temporal blocking); see acs_set_kernel */
    ACS_KERNEL_LB = 4        /* 2d+1 stored populations: collide, then stream + solve (acs_lb_bind) */
};

/* Schemes (acs_set_scheme).  RLB-MIE-FD is the paper's scheme (Eq. IE-FD); FEX-FD
 * is the fully explicit scheme Remark 2 compares against,
 * phi <- phi + lambda sum_k(...) - dt f(phi). */
enum { ACS_SCHEME_RLB_MIE_FD = 0, ACS_SCHEME_FEX_FD = 1 };

/*
 * acs_create -- validate a problem and make a context for it.
 *   dims   1, 2 or 3 (the D1Q3, D2Q5, D3Q7 lattices of Eq. ci)
 *   n      unknowns per axis, n[0..dims-1] >= 1 (entries past dims are ignored);
 *          n[dims-1] is the fastest axis.  The product must be < 2^40.
 *   eps    interfacial parameter eps > 0 of Eq. (ACE) (the equation's diffusion
 *          coefficient is eps^2); eps == 0 is accepted and gives the pure reaction flow
 *   dt     time step, 0 < dt < 2 (for dt >= 2 the cubic of Remark 1 stops being
 *          monotone and its root need not be unique)
 *   h      lattice spacing Delta x > 0
 *   bc     ACS_BC_*;  dtype ACS_F32 or ACS_F64
 * Returns ACS_OK, or ACS_WARN_MP_CONDITION / ACS_WARN_ENERGY_CONDITION when the
 * step sizes violate the conditions of Theorem 2 / Theorem 3 (the context is
 * still created: the paper runs such cases on purpose), or ACS_E_INVAL with
 * *out untouched.  Theorem 2 asks for dt <= 1 - 2 d omega1/s, 0 < omega1 <= 1/(2d),
 * s > 1 with lambda = omega1/s; the weight omega1 of the lattice model does not
 * enter the finite-difference step, and a weight with s > 1 exists whenever
 * dt <= 1 - 2 d lambda, so that is the condition checked.
 * While it holds (and |phi0| <= 1) the exact scheme keeps |phi| <= 1; the kernels
 * then round an overshoot of at most 16 units in the last place back to +-1.
 */
ACS_API int acs_create(int dims, const int64_t n[3], double eps, double dt, double h, int bc,
                       int dtype, acs_ctx** out);

/* Bytes of device work memory acs_bind() needs (one state plus scratch), or 0 for NULL. */
ACS_API size_t acs_work_bytes(const acs_ctx* ctx);

/*
 * acs_bind -- attach device memory and a stream.
 *   d_phi   the state, prod(n) elements of the context's dtype, 16-byte aligned
 *   d_work  >= acs_work_bytes() bytes, 256-byte aligned; contents are scratch
 *   stream  a cudaStream_t (NULL = the legacy default stream)
 * May be called again to rebind.  ACS_E_INVAL for NULL or misaligned pointers
 * or a short work buffer (work_bytes is its size).  Resets the step counter.
 */
ACS_API int acs_bind(acs_ctx* ctx, void* d_phi, void* d_work, size_t work_bytes, void* stream);

/* Copy an initial state into d_phi (device to device, prod(n) elements) and reset
 * the step counter; d_phi0 may equal d_phi. */
ACS_API int acs_set_state(acs_ctx* ctx, const void* d_phi0);
/* The same from host memory (pageable or pinned); returns when the copy is enqueued
 * for pinned memory and after it completes for pageable memory. */
ACS_API int acs_set_state_host(acs_ctx* ctx, const void* h_phi0);
/* Copy the current state to host memory; synchronizes the stream. */
ACS_API int acs_get_state_host(acs_ctx* ctx, void* h_phi);

/* Choose the scheme (ACS_SCHEME_*). Default ACS_SCHEME_RLB_MIE_FD. */
ACS_API int acs_set_scheme(acs_ctx* ctx, int scheme);

/*
 * acs_set_kernel -- choose the kernel variant; depth is the number of fused
 * steps per pass for ACS_KERNEL_TEMPORAL and ignored otherwise (ACS_E_INVAL outside
 * 1..8).  Temporal blocking exists for 2D grids whose rows are a multiple of 16 bytes
 * (depth 2..4, FP32 and FP64) and 3D FP32 grids with rows of an even length (depth
 * 2); a run's remainder of fewer than `depth` steps takes single steps, which round
 * identically.  ACS_E_UNSUPPORTED if the variant does not exist for this problem.
 */
ACS_API int acs_set_kernel(acs_ctx* ctx, int kernel, int depth);
/* The variant acs_step() uses (after autotuning, for ACS_KERNEL_AUTO). */
ACS_API int acs_get_kernel(const acs_ctx* ctx, int* kernel, int* depth);

/*
 * acs_get_root -- how the step solves the cubic of Remark 1 (Eq. root) for this context,
 * as the host chose it from a-priori error bounds at create / set_scheme time:
 *   *mode   ACS_ROOT_NEWTON (seeded Newton corrections), ACS_ROOT_SERIES (truncated
 *           Lagrange series), ACS_ROOT_NONE (FEX-FD: no cubic)
 *   *split  FP64 series only: 1 when its terms of order xi^13 and beyond are summed in
 *           FP32 (their effect on theta is bounded by 2^-58 for every xi the series
 *           takes), 0 otherwise.
 * Either pointer may be NULL.  ACS_E_INVAL for a NULL context.
 */
enum { ACS_ROOT_NEWTON = 0, ACS_ROOT_SERIES = 1, ACS_ROOT_NONE = 2 };
ACS_API int acs_get_root(const acs_ctx* ctx, int* mode, int* split);

/*
 * Collide-and-stream (population) form, Sec. II: Eqs. (fieq-Fi), (fneq), (RLB),
 * (pine).  A DdQ(2d+1) lattice keeps 2d+1 populations per node; one step collides
 * every node into g_k = w_k phi - ((1 - s) w_1 / s)(phi(y + c_k dt) - phi(y))
 * (g_0 = w_0 phi, s = w_1 / lambda), streams them, and solves the cubic of
 * Remark 1 for the summed value.  It is the form Eq. (IE-FD) removes; it is kept
 * to measure what the macroscopic form saves in memory and traffic.
 *
 * acs_lb_bytes  size of the population buffer: (2 dims + 1) * (prod(n) + 8192) elements;
 *               population array k (k = 0; +x, +y, +z; -x, -y, -z) starts at element
 *               k * (prod(n) + 8192) (the gap keeps the arrays off a common alignment in
 *               the memory channels).
 * acs_lb_bind   d_pop: that many bytes, 16-byte aligned, caller-owned, valid while
 *               ACS_KERNEL_LB is selected; omega1: the weight w_1 in (0, 1/(2d)],
 *               or 0 for the paper's choice (1/3, 1/5, 1/6 for d = 1, 2, 3).
 *               Then acs_set_kernel(ctx, ACS_KERNEL_LB, 1) selects the form
 *               (ACS_E_STATE before acs_lb_bind; ACS_E_UNSUPPORTED with FEX-FD).
 */
ACS_API size_t acs_lb_bytes(const acs_ctx* ctx);
ACS_API int acs_lb_bind(acs_ctx* ctx, void* d_pop, size_t bytes, double omega1);

/* Number of tile shapes (rows per thread x ring depth) the tiled kernels offer. */
ACS_API int acs_num_variants(void);

/*
 * acs_set_variant -- tile shape of the tiled kernels (0 .. acs_num_variants() - 1) and
 * the work of one CTA: z planes (3D) or 16-row blocks (2D) per CTA, 0 = chosen from
 * the occupancy.  Results do not depend on it (bit-identical states).
 */
ACS_API int acs_set_variant(acs_ctx* ctx, int variant, int chunk);
ACS_API int acs_get_variant(const acs_ctx* ctx, int* variant, int* chunk);

/*
 * acs_autotune -- time every kernel variant available for this problem on the bound
 * buffers (candidates read the state and write only the work buffer, so the state is
 * unchanged), keep the fastest, and record it in the tuning cache, a text file named
 * by $ACS_TUNE_CACHE (default $HOME/.cache/acs_tune.txt; no file if neither is set)
 * keyed by (device, dims, n, bc, dtype, scheme).  A context created with
 * ACS_KERNEL_AUTO (the default) runs it on its first acs_step for problems of at least
 * 2^20 unknowns, unless the cache already holds the key or $ACS_AUTOTUNE is "0"; call
 * it explicitly before capturing the stream into a CUDA graph.  Synchronizes.
 * *us_per_step (may be NULL) receives the winner's time per step in microseconds.
 */
ACS_API int acs_autotune(acs_ctx* ctx, double* us_per_step);

/*
 * acs_step -- advance the state by n_steps >= 0 steps of Eq. (IE-FD), in place:
 * on completion (stream order) d_phi holds phi^{n + n_steps}.  Asynchronous.
 * The launches of one call are recorded once into a CUDA graph and replayed.
 */
ACS_API int acs_step(acs_ctx* ctx, int64_t n_steps);

/* Steps taken since the last acs_bind / acs_set_state. */
ACS_API int64_t acs_steps_done(const acs_ctx* ctx);

/*
 * acs_energy -- the discrete free energy of Theorem 3 (Eq. proof2-eq0),
 *   E_h = h^d [ 1/4 sum_i (phi_i^2 - 1)^2 + eps^2/2 sum_links ((phi_j - phi_i)/h)^2 ],
 * where -Phi^T Lambda_{dx} Phi is written as the sum over lattice links (periodic:
 * the wrap-around link counts; Neumann: interior links only; Dirichlet: also the
 * link from each boundary unknown to the zero boundary value).  FP64 result; the
 * sums are formed as described at ACS_F32 / ACS_F64 and combined exactly, so the
 * value is deterministic.  Synchronizes the stream.
 * ACS_E_NONFINITE (value still written) if the result is not finite.
 */
ACS_API int acs_energy(acs_ctx* ctx, double* out_host);

/* max_i |phi_i| (Theorem 2's discrete maximum norm); NaN if any entry is NaN.
 * Synchronizes the stream; ACS_E_NONFINITE (value still written) for NaN/Inf. */
ACS_API int acs_maxnorm(acs_ctx* ctx, double* out_host);

/*
 * acs_phase_volume -- the volume (area in 2D, length in 1D) of the phase phi > 0,
 * measured as h^d sum_i (1 + phi_i) / 2 over the unknowns: the quantity behind the
 * radius of the shrinking circle / sphere of Sec. IV.B.2 (motion by mean curvature,
 * R(t) = sqrt(R0^2 - 2 eps^2 t) in 2D, sqrt(R0^2 - 4 eps^2 t) in 3D).  FP64, compensated;
 * synchronizes the stream.
 */
ACS_API int acs_phase_volume(acs_ctx* ctx, double* out_host);

/* Both reductions, written as {E_h, max|phi|} to two doubles of device memory,
 * asynchronously (no synchronization). */
ACS_API int acs_observe_async(acs_ctx* ctx, double* d_out2);

/*
 * acs_run_logged -- n_steps steps with E_h and max|phi| recorded before the first
 * step and after every `every` steps (every >= 1): n_steps/every + 1 entries into
 * each host array.  One synchronization at the end.  The log lives in the work
 * buffer (at most 4096 entries per call; ACS_E_INVAL beyond).
 */
ACS_API int acs_run_logged(acs_ctx* ctx, int64_t n_steps, int64_t every, double* h_energy,
                           double* h_maxnorm);

/*
 * Adjoint of the discrete stepper (the transpose of the Jacobian of each step of
 * Eq. IE-FD, chained backwards), for a terminal loss L(phi_T):
 *   per step, mu = lambda^{n+1} / (1 + (dt/2) f'(phi^{n+1})),  f'(x) = 3x^2 - 1,
 *   lambda^n = mu (1 - (dt/2) f'(phi^n)) + lambda_lat S^T mu  (S = the ghost-rule stencil),
 *   dL/d(eps^2) += (dt/h^2) sum_i mu_i S_i(phi^n)   (dt and h held fixed).
 * Recording: acs_grad_bind() gives the context a checkpoint buffer of
 * acs_grad_work_bytes(ctx, max_steps, every) bytes; from then on acs_set_state
 * stores phi^0 and acs_step stores every `every`-th state.  acs_grad() then
 * recomputes each segment from its checkpoint and sweeps backwards over all steps
 * since acs_set_state (with every = 1 each step writes straight into its checkpoint
 * slot and nothing is recomputed: max_steps + 1 states of memory for about a quarter
 * less work), given d_dL_dphiT (the state's dtype), writing dL/dphi0 to
 * d_dL_dphi0 (same dtype; may alias d_dL_dphiT) and dL/d(eps^2) (accumulated in
 * FP64) to *dL_deps2_host.  Synchronizes.  ACS_E_STATE if nothing was recorded,
 * ACS_E_NOMEM if more than max_steps steps were taken.
 */
ACS_API size_t acs_grad_work_bytes(const acs_ctx* ctx, int64_t max_steps, int64_t every);
ACS_API int acs_grad_bind(acs_ctx* ctx, void* d_grad_work, size_t bytes, int64_t max_steps,
                          int64_t every);
ACS_API int acs_grad(acs_ctx* ctx, const void* d_dL_dphiT, void* d_dL_dphi0, double* dL_deps2_host);

/*
 * acs_observe_noalloc -- {E_h, max|phi|} of a state, like acs_observe_async, for
 * callers that cannot allocate device memory (the paper has no counterpart: this is
 * a deployment aid).  Some callers have no work buffer and cannot make one: code
 * that must not call cudaMalloc because it can synchronize the device, plugins
 * whose host application owns all device memory through its own pool, and tools
 * that only hold a pointer to someone else's state.  This call needs no context and
 * allocates nothing: its scratch is a 64 KiB array of static device memory that
 * the library holds on every GPU that loads it, until the process exits.
 *   dims, n, eps, h, bc, dtype  the problem, as for acs_create (dt is not needed)
 *   d_phi    the state in device memory (prod(n) elements of dtype)
 *   d_out2   two doubles of device memory receiving {E_h, max|phi|}
 *   stream   the cudaStream_t to run on (NULL = legacy default stream)
 * Asynchronous.  Shapes beyond acs_create's limit (2^40 elements) are rejected with
 * ACS_E_INVAL, as are NULL or misaligned pointers.  The first call on a device looks
 * up the array's device address (cudaGetSymbolAddress); make that first call before
 * any stream capture begins.  Every call shares the one array and it keeps the last
 * call's partial sums; each call overwrites every entry it reads, so nothing needs
 * clearing, but calls whose kernels overlap on the GPU (other streams, other host
 * threads) race on it: order them on one stream or synchronize between them.
 */
ACS_API int acs_observe_noalloc(int dims, const int64_t n[3], double eps, double h, int bc, int dtype,
                                const void* d_phi, double* d_out2, void* stream);

/* Block until all work enqueued by this context has finished. */
ACS_API int acs_sync(acs_ctx* ctx);

/*
 * acs_dt_max -- the step-size bounds of the paper for lattice number lambda =
 * eps^2 dt / h^2 on the DdQ(2d+1) lattice:
 *   *dt_mp      largest dt with dt <= 1 - 2 d lambda                     (Theorem 2)
 *   *dt_energy  largest dt with dt <= 4 (1 - 2 d lambda)                 (Theorem 3)
 */
ACS_API int acs_dt_max(int dims, double eps, double h, double* dt_mp, double* dt_energy);

/* Human-readable text of a status code (static storage). */
ACS_API const char* acs_strerror(int status);

/* Library version as "major.minor.patch" (static storage). */
ACS_API const char* acs_version(void);

/* Release the context (not the caller's buffers).  Waits for its stream. NULL is a no-op. */
ACS_API void acs_destroy(acs_ctx* ctx);

/*
 * Batched stepping: `count` independent 2D problems of sides n[i] x n[i], each
 * with its own eps, dt, h and boundary (Sec. I, Eq. IE-FD), advanced together in
 * one persistent launch per call (recorded into a CUDA graph).  The paper has no
 * batched form; this is many copies of the 2D step.
 *
 * Layout: the states are packed one after the other in one device buffer of
 * acs_batch_numel() elements.  Instance i starts at element offsets[i]
 * (acs_batch_offsets) and its rows are row_strides[i] elements apart
 * (acs_batch_row_strides: n[i] rounded up to a multiple of 16 bytes); row y,
 * column x of instance i is element offsets[i] + y * row_strides[i] + x.  The
 * padding after each row is never read into a result nor written.
 *
 * Per-instance arithmetic is identical to acs_step() on that instance alone, so
 * each instance's state is bit-identical to its standalone run.
 *
 * acs_batch_create  validates every instance (as acs_create) and plans the work;
 *                   returns the strongest ACS_WARN_* over the instances, or an error
 *                   (ACS_E_INVAL) with *out untouched.  The caller owns *out
 *                   (acs_batch_destroy).
 * acs_batch_bind    d_phi: the packed states (16-byte aligned, caller-owned, stays
 *                   valid while bound); d_work: acs_batch_work_bytes() bytes, 256-byte
 *                   aligned, caller-owned; stream: where every call is enqueued.
 *                   ACS_E_UNSUPPORTED if the TMA descriptors cannot be encoded.
 * acs_batch_step    advances every instance n_steps (asynchronous on the stream).
 */
ACS_API int acs_batch_create(int count, const int64_t* n, const double* eps, const double* dt,
                             const double* h, const int* bc, int dtype, acs_batch** out);
ACS_API size_t acs_batch_numel(const acs_batch* b);
ACS_API int acs_batch_offsets(const acs_batch* b, int64_t* offsets);
/* Row stride (elements) of every instance into `count` int64 values. */
ACS_API int acs_batch_row_strides(const acs_batch* b, int64_t* row_strides);
ACS_API size_t acs_batch_work_bytes(const acs_batch* b);
ACS_API int acs_batch_bind(acs_batch* b, void* d_phi, void* d_work, size_t work_bytes, void* stream);
ACS_API int acs_batch_step(acs_batch* b, int64_t n_steps);

/*
 * Launch configuration of the batched kernel (results do not depend on it: every
 * instance stays bit-identical to its standalone run).
 *   ctas_per_sm        CTAs of the persistent grid per SM, 0 = as many as fit
 *                      (acs_batch_get_config then reports that number once bound)
 *   blocks_per_ticket  consecutive blocks a CTA takes per draw, 1..16
 *   order              0: blocks instance after instance; 1: the largest instances'
 *                      blocks first (the small ones then fill the end of each step)
 * acs_batch_set_config  ACS_E_INVAL for values outside those ranges.
 * acs_batch_autotune    times every (ctas_per_sm, blocks_per_ticket in {1, 2, 4},
 *                       order) of the single-step kernel and, where the batch can use
 *                       temporal blocking, every (depth 2..4, rows_per_unit in {32, 64,
 *                       128}, order) of the temporally blocked kernel, on the bound batch
 *                       with launches of about 16 steps in which every step (pass) reads
 *                       the state and writes the work buffer's second state (the state
 *                       is unchanged); keeps the fastest (the single-step kernel's best
 *                       configuration stays set for the steps a temporal block leaves
 *                       over) and records it in the tuning cache (see acs_autotune) under
 *                       the batch's workload class: dtype, instance count, total
 *                       unknowns, a histogram of sides in octaves and the boundary mix.
 *                       acs_batch_bind applies a cached choice for the class.
 *                       Synchronizes; *us_per_step (may be NULL) receives the winner's
 *                       time per step.  ACS_E_STATE before acs_batch_bind.
 * The paper has no batched form; this tunes the launch of many copies of its 2D step.
 */
ACS_API int acs_batch_set_config(acs_batch* b, int ctas_per_sm, int blocks_per_ticket, int order);
ACS_API int acs_batch_get_config(const acs_batch* b, int* ctas_per_sm, int* blocks_per_ticket, int* order);
ACS_API int acs_batch_autotune(acs_batch* b, double* us_per_step);

/*
 * Temporal blocking of the batched form: K = depth steps of Eq. IE-FD per pass
 * through HBM, in one persistent launch for all passes of an acs_batch_step call
 * (nsteps / K passes, then nsteps % K single steps).  Each instance is cut into units
 * of a 120-column strip by a chunk of at most rows_per_unit rows (balanced over the
 * side); a unit recomputes K cells of halo at each side, so its state after a pass is
 * bit-identical to K single steps.  Units of a pass wait (bounded) only for their own
 * instance's previous pass, not for a grid barrier.
 *   depth          1 = the single-step kernel only; 2..4
 *   rows_per_unit  0 = the default (64), else 16 .. 2^20
 *   order          0: units instance after instance; 1: the largest instances' units
 *                  first (the single-step kernel keeps its own order, acs_batch_set_config)
 * acs_batch_set_temporal  ACS_E_INVAL outside those ranges; ACS_E_UNSUPPORTED for
 *                         depth >= 2 on an FP64 batch (the FP64 step is bound by the
 *                         FP64 pipe, not by HBM).  Applies on the next acs_batch_step;
 *                         needs no rebinding.
 * acs_batch_get_temporal  the depth, rows per unit and unit order in effect (any may be
 *                         NULL).
 * Results do not depend on the setting.  The paper has no batched form.
 */
ACS_API int acs_batch_set_temporal(acs_batch* b, int depth, int rows_per_unit, int order);
ACS_API int acs_batch_get_temporal(const acs_batch* b, int* depth, int* rows_per_unit, int* order);
/* Per-instance E_h and max|phi| into host arrays of `count` doubles; synchronizes. */
ACS_API int acs_batch_observe(acs_batch* b, double* h_energy, double* h_maxnorm);
/* Testing aid for the failure path: mode 1 makes one CTA of the next single-step
 * batched launch skip its arrival at the first step barrier (with temporal blocking:
 * the completion of the launch's first unit goes uncounted), so the other CTAs'
 * (warps') bounded waits (about one second) expire, the launch ends early, and the
 * next acs_batch_observe returns ACS_E_TIMEOUT (which also clears the fault state);
 * mode 0 disarms it.  No GPU fault is involved. */
ACS_API int acs_batch_inject_fault(acs_batch* b, int mode);
ACS_API void acs_batch_destroy(acs_batch* b);

/*
 * Batched lines: `count` independent 1D problems (Eq. IE-FD with d = 1) of n[i]
 * unknowns, each with its own eps, dt, h and boundary (Eq. Ddeltax at both ends).  The
 * paper's 1D runs (Table 2, Fig. 4) are such lines; this is many of them at once.  A
 * line of up to 1024 unknowns (FP64: 512) is held in one warp's registers and a longer
 * one (up to 28672, FP64 14336) in one CTA's shared memory for all the steps of a call,
 * so the state touches device memory only at the call's start and end; lines of
 * different size classes run concurrently.  Each line's state is bit-identical to
 * acs_step() on that line alone.
 *
 * Layout: line i is the n[i] values at element offsets[i] (acs_lines_offsets) of one
 * device buffer of acs_lines_numel() elements; lines start on 16-byte boundaries.
 *
 * acs_lines_create  validates every line as acs_create does (dims = 1) and rejects
 *                   lines longer than the limits above (ACS_E_INVAL; acs_step handles
 *                   those); returns the strongest ACS_WARN_* over the lines.  The
 *                   caller owns *out (acs_lines_destroy).
 * acs_lines_bind    d_phi: the packed states (16-byte aligned); d_work:
 *                   acs_lines_work_bytes() bytes, 256-byte aligned; both caller-owned and
 *                   valid while bound; stream: where every call is enqueued.
 * acs_lines_step    advances every line n_steps (asynchronous on the stream).
 * acs_lines_observe per-line E_h and max|phi| into host arrays of `count` doubles
 *                   (synchronizes).
 */
ACS_API int acs_lines_create(int count, const int64_t* n, const double* eps, const double* dt,
                             const double* h, const int* bc, int dtype, acs_lines** out);
ACS_API size_t acs_lines_numel(const acs_lines* L);
ACS_API int acs_lines_offsets(const acs_lines* L, int64_t* offsets);
ACS_API size_t acs_lines_work_bytes(const acs_lines* L);
ACS_API int acs_lines_bind(acs_lines* L, void* d_phi, void* d_work, size_t work_bytes, void* stream);
ACS_API int acs_lines_step(acs_lines* L, int64_t n_steps);
ACS_API int acs_lines_observe(acs_lines* L, double* h_energy, double* h_maxnorm);
ACS_API void acs_lines_destroy(acs_lines* L);

/*
 * Pipelined host-to-host runs: a stream of independent jobs, each "copy phi^0 from
 * host memory, advance n_steps steps of Eq. IE-FD (logging E_h and max|phi| every
 * `every` steps, as acs_run_logged), copy phi^N back to host memory".  `slots` device
 * states (2 to 4) take consecutive jobs in turn, so the host-to-device copy of a later
 * job and the device-to-host copy of an earlier one run on their own streams while a
 * job computes on the bound stream.  Every job's results are those of
 * acs_set_state_host, acs_run_logged and acs_get_state_host on one context, bit for bit.
 *
 * acs_pipe_create   validates as acs_create does (and 2 <= slots <= 4, else
 *                   ACS_E_INVAL) and returns its status; the caller owns *out
 *                   (acs_pipe_destroy).  Host-only (no CUDA call).
 * acs_pipe_bytes    device bytes acs_pipe_bind needs: one state and one work area
 *                   (acs_work_bytes) per slot, each rounded up to 256 bytes.
 * acs_pipe_bind     d_buf: acs_pipe_bytes() bytes of device memory, 256-byte aligned,
 *                   caller-owned and valid while bound; stream: where the steps run.
 *                   Creates the two copy streams and the events the library owns.
 * acs_pipe_context  slot in [0, slots): the context that runs that slot's jobs, for
 *                   acs_set_kernel / acs_set_scheme / acs_set_variant (apply the same
 *                   setting to every slot).  Owned by the pipe; never destroy or rebind it.
 * acs_pipe_submit   enqueues one job and returns without waiting.  h_in (read) and
 *                   h_out (written): n[0] x ... x n[dims-1] values of the dtype;
 *                   h_log: 2 (n_steps / every + 1) doubles {E_h, max|phi|} per entry, or
 *                   null with every = 0 (no logging; ACS_E_INVAL if every < 0, or if
 *                   h_log is null while every > 0, or more than 4096 entries).  The
 *                   host buffers must stay valid and untouched until acs_pipe_wait
 *                   returns; page-locked buffers are what lets the copies overlap
 *                   (pageable ones work, serialized).
 * acs_pipe_wait     waits for every submitted job; ACS_E_TIMEOUT if a kernel's bounded
 *                   wait gave up, ACS_E_NONFINITE if a logged value is NaN/Inf (the
 *                   outputs are still written), else ACS_OK.
 */
ACS_API int acs_pipe_create(int dims, const int64_t n[3], double eps, double dt, double h, int bc, int dtype,
                            int slots, acs_pipe** out);
ACS_API size_t acs_pipe_bytes(const acs_pipe* p);
ACS_API int acs_pipe_bind(acs_pipe* p, void* d_buf, size_t bytes, void* stream);
ACS_API acs_ctx* acs_pipe_context(acs_pipe* p, int slot);
ACS_API int acs_pipe_submit(acs_pipe* p, const void* h_in, void* h_out, int64_t n_steps, int64_t every,
                            double* h_log);
ACS_API int acs_pipe_wait(acs_pipe* p);
ACS_API void acs_pipe_destroy(acs_pipe* p);

#ifdef __cplusplus
}
#endif

#endif /* ACS_H */
