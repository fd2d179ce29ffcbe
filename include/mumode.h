/*
 * mumode.h -- C ABI of the B300 mu-mode integrator library (libmumode.so).
 *
 * The library applies the mu-mode integrator of Caliari, Cassini, Einkemmer,
 * Ostermann and Zivcovich (arXiv 2103.01691) on one GPU: the Tucker operator
 * U x_1 E_1 x_2 E_2 ... x_d E_d with precomputed one-dimensional
 * exponentials E_mu = exp(tau A_mu) (section 2, eq. (dd-tensor)), Hermite
 * spectral transforms written as mu-mode products (section 3, eqs.
 * (real2spec) and (spec2real)), and the Strang splitting step of the cubic
 * nonlinear Schroedinger / Gross-Pitaevskii equation (section 4.5).
 *
 * Conventions shared by every call
 * --------------------------------
 * Tensor layout.  A d-way tensor with sizes n[0..d-1] = (n_1, ..., n_d) is
 *   stored with i_1 fastest: element (i_1, ..., i_d) (0-based) lives at
 *   i_1 + n_1 (i_2 + n_2 (i_3 + ...)) (section 4.1, after eq. (exactsol)).
 *   A torch tensor of shape (n_d, ..., n_1), contiguous, has this layout.
 * Matrices.  Host matrices are row-major FP64.  Complex host matrices are
 *   interleaved (re, im) pairs: entry (i, j) of an m x n complex matrix is
 *   at [2 (i n + j)] (re) and [2 (i n + j) + 1] (im).
 * Complex device data.  MM_C64 is interleaved (re, im) float32 pairs,
 *   MM_C128 interleaved float64 pairs.
 * Ownership.  The caller owns every pointer it passes.  *_dev pointers are
 *   device memory of the context's device, 16-byte aligned, holding the
 *   full tensor contiguously.  Plans own their device copies of the
 *   matrices and their workspace.
 * Streams.  `stream` is a cudaStream_t passed as void*; NULL is the legacy
 *   default stream.  Calls enqueue work and return without synchronising
 *   unless stated.
 * Errors.  Every call returns mm_status.  Arguments are checked before
 *   any work is enqueued; on failure nothing is launched and
 *   mm_last_error() (thread-local) describes the problem.  Device-side
 *   bounded waits never hang: when one gives up the kernel records
 *   MM_ERR_TIMEOUT in the context's device error word, which
 *   mm_device_status() reads.  Nothing aborts or traps.
 */
#ifndef MUMODE_H
#define MUMODE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mm_ctx mm_ctx;
typedef struct mm_plan mm_plan;

typedef enum {
    MM_OK = 0,
    MM_ERR_INVALID_ARG = 1, /* null pointer, bad index or value */
    MM_ERR_SHAPE = 2,       /* sizes outside what the chosen path supports */
    MM_ERR_DTYPE = 3,       /* dtype / precision combination not supported */
    MM_ERR_ALIGN = 4,       /* device pointer not 16-byte aligned */
    MM_ERR_OOM = 5,         /* device allocation failed */
    MM_ERR_CUDA = 6,        /* a CUDA runtime call failed */
    MM_ERR_TIMEOUT = 7,     /* a device-side bounded wait gave up */
    MM_ERR_UNSUPPORTED = 8, /* feature not available on this device */
    MM_ERR_RANGE = 9        /* MM_PREC_F16X6: the state grew more than 16x within
                               one sweep, beyond its fixed-point range */
} mm_status;

typedef enum {
    MM_R64 = 0,  /* real float64 */
    MM_C64 = 1,  /* complex float32 (interleaved) */
    MM_C128 = 2, /* complex float64 (interleaved) */
    MM_R32 = 3   /* real float32 */
} mm_dtype;

/* Arithmetic of the mode contractions.
 * MM_PREC_FP64_SIMT  FP64 FMA on CUDA cores; state MM_R64 or MM_C128.
 * MM_PREC_FP32_SIMT  FP32 FMA on CUDA cores; state MM_R32 or MM_C64.
 * MM_PREC_BF16X6     tcgen05 tensor cores, state MM_C64.  Matrix and state
 *                    are split into three BF16 pieces (x = x0 + x1 + x2,
 *                    exact for FP32 x), the six products with piece
 *                    orders a + b <= 2 are summed in FP32 in tensor memory,
 *                    the leading product in an accumulator of its own.
 * MM_PREC_BF16X3     as above with two pieces and the three products
 *                    a + b <= 1.
 * MM_PREC_BF16       one BF16 piece, one product (reported, not accurate).
 * MM_PREC_F16X6      tcgen05 tensor cores, state MM_C64, the accurate split
 *                    mode.  The tensor cores truncate when they add to an
 *                    FP32 accumulator, which biases long runs of the BF16
 *                    modes.  Here the leading pieces are integers on
 *                    power-of-two grids (a scale per matrix row, and one
 *                    per state tensor that follows the state's maximum from
 *                    sweep to sweep), so the leading product is summed
 *                    exactly; two FP16 pieces carry the remainders and the
 *                    five correction products go to a second accumulator.
 *                    Relative L2 error <= 1e-6 after 50 steps at n = 256.
 * MM_PREC_FP64_DMMA  FP64 on the tensor cores through the warp-level MMA
 *                    (m8n8k4, the only FP64 MMA form; tcgen05 has no FP64
 *                    kind); state MM_R64 or MM_C128, same accuracy as
 *                    MM_PREC_FP64_SIMT.
 * MM_PREC_AUTO       chosen from the data type and sizes when the plan or
 *                    product is created: MM_C64 -> MM_PREC_F16X6 when every
 *                    n_mu (and m) is at most 512, else MM_PREC_FP32_SIMT;
 *                    MM_R32 -> MM_PREC_FP32_SIMT; MM_R64, MM_C128 ->
 *                    MM_PREC_FP64_DMMA.
 * MM_PREC_TF32X3     "3xTF32": tcgen05 tensor cores (kind::tf32), state
 *                    MM_C64.  Matrix and state are split into two TF32
 *                    pieces each (x0 = TF32 of x, x1 = TF32 of x - x0, both
 *                    rounded to nearest even; about 22 bits together), and
 *                    the three products e0 x0, e0 x1, e1 x0 are summed in
 *                    FP32 in tensor memory, the leading one in an
 *                    accumulator of its own.  The tensor cores truncate
 *                    when they add to an FP32 accumulator, so the floating
 *                    pieces carry a bias, as in MM_PREC_BF16X6; the
 *                    precision sweep reports its error.  Tucker plans and
 *                    mumode_product only (the one-SM kernel); other calls
 *                    return MM_ERR_UNSUPPORTED. */
typedef enum {
    MM_PREC_FP64_SIMT = 0,
    MM_PREC_FP32_SIMT = 1,
    MM_PREC_BF16X6 = 2,
    MM_PREC_BF16X3 = 3,
    MM_PREC_BF16 = 4,
    MM_PREC_F16X6 = 5,
    MM_PREC_FP64_DMMA = 6,
    MM_PREC_AUTO = 7,
    MM_PREC_TF32X3 = 8
} mm_prec;

/* ---------------------------------------------------------------------
 * Context
 * ------------------------------------------------------------------- */

/* Create a context on CUDA device `device` (makes it current for the
 * calling thread).  Allocates a small device error word.  *out receives
 * the context.  Errors: MM_ERR_INVALID_ARG (out NULL or bad device),
 * MM_ERR_CUDA, MM_ERR_UNSUPPORTED (device is not sm_103). */
mm_status mm_ctx_create(int device, mm_ctx **out);
void mm_ctx_destroy(mm_ctx *ctx);

/* Thread-local description of the last failure (never NULL). */
const char *mm_last_error(void);

/* Synchronise `stream`, read and clear the context's device error word.
 * Returns MM_OK, MM_ERR_TIMEOUT (a bounded device wait gave up) or
 * MM_ERR_CUDA (a kernel or copy failed). */
mm_status mm_device_status(mm_ctx *ctx, void *stream);

/* Number of kernels this library has launched in the calling process
 * (all contexts), for launch accounting. */
int64_t mm_launch_count(void);

/* Kernel timing (tracing aid, not from the paper).  While enabled, every
 * mode-product kernel launched through `ctx` is bracketed by a pair of CUDA
 * events on its stream.  mm_kernel_timing_read() waits for the recorded
 * events, returns the summed kernel time in milliseconds and the number of
 * timed launches, and starts a new record.  Enabling also clears the
 * record.  Errors: MM_ERR_INVALID_ARG for NULL arguments, MM_ERR_CUDA. */
mm_status mm_kernel_timing(mm_ctx *ctx, int enable);
mm_status mm_kernel_timing_read(mm_ctx *ctx, double *total_ms, int64_t *launches);

/* ---------------------------------------------------------------------
 * Host set-up in FP64 (section 2: the d small exponentials are computed
 * once for a constant step; section 4.1: expm by scaling and squaring).
 * ------------------------------------------------------------------- */

/* Centered second-order FD Laplacian with homogeneous Dirichlet conditions
 * on (0,1), interior nodes x_j = j/(n+1): A = (n+1)^2 tridiag(1,-2,1),
 * n x n row-major into A_out (caller-allocated, n*n doubles). */
mm_status mm_fd_laplacian_dirichlet(int n, double *A_out);

/* E = exp(z A) in FP64 for an n x n matrix A (real part A_re, imaginary
 * part A_im or NULL) and a complex scalar z = z_re + i z_im, by scaling and
 * squaring with the degree-13 Pade approximant (Higham 2005).  E_out is an
 * n x n complex matrix (2*n*n doubles, interleaved), caller-allocated. */
mm_status mm_expm(int n, const double *A_re, const double *A_im, double z_re, double z_im,
                  double *E_out);

/* Gauss-Hermite rule with m nodes (section 3, eq. (quadrature); the nodes
 * make the Hermite functions discretely orthonormal).  x_out: nodes
 * ascending; W_out: weights for plain integrals, sum_l W_l f(x_l) ~ int f,
 * i.e. the Gauss weights for exp(-x^2) times exp(x_l^2).  Computed as the
 * eigenvalues of the Jacobi matrix (Golub-Welsch) by Sturm bisection, then
 * W_l = 1 / sum_{k<m} phi_k(x_l)^2.  Both arrays hold m doubles. */
mm_status mm_gauss_hermite(int m, double *x_out, double *W_out);

/* Hermite-function matrices at the m Gauss-Hermite nodes (section 3):
 * fwd[k][l] = phi_k(x_l) W_l   (values -> coefficients, eq. (real2spec)
 *                               with the weights folded in),
 * bwd[l][k] = phi_k(x_l)       (coefficients -> values, eq. (spec2real),
 *                               Psi = Phi^*).
 * Either output may be NULL.  m x m doubles each, row-major. */
mm_status mm_hermite_matrices(int m, double *fwd, double *bwd);

/* ---------------------------------------------------------------------
 * mu-mode product (Definition 2.1): S = U x_mu L.
 * d in 1..8, n[0..d-1] the sizes of U, mu in 1..d, L an m x n_mu matrix
 * (FP64 host, complex interleaved if L_is_complex), S has n_mu replaced by
 * m.  u_dev and s_dev must not overlap.  dtype / prec:
 *   MM_PREC_FP64_SIMT with MM_C128 (or MM_R64 if L is real),
 *   MM_PREC_FP32_SIMT with MM_C64 (or MM_R32 if L is real),
 *   MM_PREC_BF16* with MM_C64; tensor-core paths need n_mu, m <= 512.
 * The matrix is uploaded on every call (use a plan for repeated use);
 * the call allocates and frees its temporaries, so it synchronises the
 * stream before returning.
 * ------------------------------------------------------------------- */
mm_status mumode_product(mm_ctx *ctx, int d, const int64_t *n, int mu, const double *L,
                         int64_t m, int L_is_complex, mm_dtype dtype, mm_prec prec,
                         const void *u_dev, void *s_dev, void *stream);

/* The paper has no counterpart to this call: it is a service for callers
 * that cannot allocate device memory.  Examples are code running under a
 * framework whose caching allocator already owns the GPU's memory (a
 * cudaMalloc there either fails or fragments the pool), latency-critical
 * loops that cannot afford cudaMalloc's implicit device synchronisation,
 * and plugins whose host forbids device allocation.
 *
 * mumode_product_noalloc computes what mumode_product computes with
 * MM_PREC_F16X6 on MM_C64 data, on the current CUDA device, with no device
 * allocation: it calls no cudaMalloc, cudaFree or other routine that
 * allocates device memory.  (The matrix pieces are built on the host in
 * ordinary host memory, as in mumode_product.)  The caller passes the
 * input u_dev and the output s_dev as in mumode_product.  All temporaries
 * (the split input and output states, the matrix pieces, the scale and
 * status words) live in one static device array of 64 MiB that every GPU
 * loading this library reserves until the process exits.  A product fits
 * when about 12 bytes per padded input point plus 12 per padded output
 * point plus ~1.2 MB for the matrix stay within 64 MiB (for example
 * 128^3 points); larger products are rejected with MM_ERR_SHAPE before
 * anything is enqueued.  n_mu and m must be at most 256.
 *
 * Every call uses the same array, and the array keeps the previous call's
 * contents; the call clears the words that must start at zero itself.
 * Calls whose work overlaps on the GPU (other threads, other streams) race
 * on the array: serialise them.  The first call on each device looks up
 * the array's device address (cudaGetSymbolAddress) with that device
 * current; make that first call before any stream capture.  The call
 * synchronises `stream` before returning and reports device-side checks
 * (MM_ERR_TIMEOUT, MM_ERR_RANGE) in its status. */
mm_status mumode_product_noalloc(int d, const int64_t *n, int mu, const double *L, int64_t m,
                                 int L_is_complex, const void *u_dev, void *s_dev, void *stream);

/* ---------------------------------------------------------------------
 * Device exponentials and matrices that change between steps (section
 * 4.4: with a time-dependent operator the exponentials change every step,
 * so they are computed on the GPU as well).
 * ------------------------------------------------------------------- */

/* E = exp(z (A + f B)) in FP64 on the device (for real z the same
 * series in real arithmetic).  A_dev, B_dev: real n x n,
 * row-major, device (B_dev may be NULL); E_dev: n x n complex interleaved
 * (2 n^2 doubles), device, overlapping neither.  Scaling and squaring of
 * the degree-18 Taylor polynomial (Paterson-Stockmeyer evaluation; the
 * products are cuBLAS ZGEMMs).  For a purely imaginary z = i w the call
 * computes cos(w M) + i sin(w M), M = A + f B, instead: degree-9
 * polynomials in (w M / 2^s)^2 and s angle doublings, all in real
 * arithmetic (the library's own FP64 tensor-core GEMM, warp MMA), about a
 * third of the flops; real z also runs on that GEMM.
 * norm_bound >= ||A + f B||_1 picks the
 * scaling; norm_bound <= 0 has the call compute the norm on the device and
 * synchronise the stream.  Otherwise stream-ordered.  Calls on one context
 * share its workspace (allocated on first use): serialise them.
 * Errors: MM_ERR_SHAPE for n outside 1..4096, MM_ERR_INVALID_ARG,
 * MM_ERR_OOM, MM_ERR_CUDA. */
mm_status mm_expm_device(mm_ctx *ctx, int n, const double *A_dev, const double *B_dev, double f, double z_re,
                         double z_im, double norm_bound, double *E_dev, void *stream);

/* Replace direction mu's matrix of a Tucker plan by E_dev (n_mu x n_mu
 * complex interleaved FP64, row-major, device memory), in stream order:
 * the plan's later steps use it.  Tensor-core plans split it into their
 * pieces on the device (from then on no k-block of that direction is
 * skipped); FP64 plans (MM_C128) copy it.  row_norm_bound >= max_i sum_j
 * |E_ij| bounds the first product of a step call (fixed-point scaling);
 * row_norm_bound <= 0 has the call read E back to compute it (synchronising
 * the stream).  Errors: MM_ERR_INVALID_ARG (Hermite plan, mu outside 1..d),
 * MM_ERR_DTYPE (FP32 or real SIMT plans), MM_ERR_CUDA. */
mm_status mm_plan_set_matrix_device(mm_plan *plan, int mu, const double *E_dev, double row_norm_bound,
                                    void *stream);

/* ---------------------------------------------------------------------
 * Pipe flow (section 4.2): c_t = alpha (c_rr + c_r / r + c_zz) - s(z) c_z
 * on [r_min, r_max] x [0, z_max], radially symmetric, centred second-order
 * differences; a Kronecker sum of a radial and an axial operator, so the
 * exact solution at T is the Tucker operator of exp(T A_r), exp(T A_z).
 * Grids: r_j = r_min + j (r_max - r_min)/(n_r - 1), j < n_r, with c_r = 0
 * at both ends (mirrored neighbour); z_j = j z_max / n_z, j = 1..n_z, with
 * c = 0 at z = 0 (not an unknown) and c_z = 0 at z_max (mirrored).
 *
 * mm_pipe_operators: A_r (n_r x n_r) and A_z (n_z x n_z), row-major, host,
 * caller-allocated (either may be NULL); s_nodes[j] = s(z_{j+1}) (n_z
 * values, or NULL for no advection).
 *
 * pipe_plan_create: a d = 2 Tucker plan (real MM_R64 data, direction 1 = r,
 * fastest) whose step is the solution operator over T: the operators as
 * above, exp(T A) of each on the device (mm_expm_device, real series),
 * FP64 precisions only (MM_PREC_FP64_SIMT, MM_PREC_FP64_DMMA; any n).
 * Synchronises the default stream. */
mm_status mm_pipe_operators(int n_r, int n_z, double rmin, double rmax, double zmax, double alpha,
                            const double *s_nodes, double *A_r, double *A_z);
mm_status pipe_plan_create(mm_ctx *ctx, int n_r, int n_z, double rmin, double rmax, double zmax, double alpha,
                           const double *s_nodes, double T, mm_prec prec, mm_plan **out);

/* ---------------------------------------------------------------------
 * Tucker-operator plan: U <- U x_{o_1} E_{o_1} ... x_{o_d} E_{o_d}
 * (section 2, eq. (dd-tensor)), repeated nsteps times (a marching scheme
 * with constant step).  E_host[mu-1] is the n_mu x n_mu matrix for
 * direction mu (complex interleaved if E_is_complex).  mode_order lists
 * the directions (1-based) in application order; NULL means 1..d.  The
 * factors commute mathematically; the order only changes rounding.
 * The plan uploads the matrices in the form the precision needs and
 * allocates its workspace (two state-sized buffers).
 * ------------------------------------------------------------------- */
mm_status mumode_plan_create(mm_ctx *ctx, int d, const int64_t *n, const double *const *E_host,
                             int E_is_complex, mm_dtype dtype, mm_prec prec,
                             const int *mode_order, mm_plan **out);

/* nsteps applications of the plan's Tucker operator to u_dev, in place. */
mm_status mumode_step(mm_plan *plan, void *u_dev, int64_t nsteps, void *stream);

/* The same on a HOST tensor (u_host, pinned or pageable): copies it to the
 * plan's device staging buffer, steps, copies the result back, and
 * synchronises the stream. */
mm_status mumode_step_host(mm_plan *plan, void *u_host, int64_t nsteps, void *stream);

void mm_plan_destroy(mm_plan *plan);

/* Autotuner (the project's own): times every kernel variant (tensor-core
 * plans: 0 = CTA pair with row tiles of at most 64, 1 = CTA pair with row
 * tiles of at most 128, 2 = one SM) and, for Tucker plans with d <= 4,
 * every mode order, nsteps steps each (1..1000, after one warm step) on a
 * scratch copy of u_dev (which is left unchanged), in two passes whose
 * faster time counts (the first pass also brings an idle GPU to its
 * clocks), and keeps the fastest in the plan.  Hermite plans time harmonic-oscillator steps and keep their
 * mode order.  Allocates a state-sized scratch for the call.
 * Cache (not from the paper): when the environment variable
 * MM_AUTOTUNE_CACHE names a file, a plan whose key is in it takes the
 * stored variant and order without timing anything (u_dev is not read),
 * and a new result is appended as one JSON line {"key": ..., "variant":
 * v, "order": [...]}.  The key holds the step kind (steps or GPE steps),
 * the GPU's name, the plan kind, sizes, dtype, precision and, for
 * tensor-core Tucker plans, a hash of the matrices' k-block bands.
 * Errors: MM_ERR_INVALID_ARG, MM_ERR_OOM, and those of the timed steps (the
 * plan's configuration is then unchanged). */
mm_status mm_plan_autotune(mm_plan *plan, const void *u_dev, int64_t nsteps, void *stream);
/* The plan's kernel variant and mode order (order_out: d ints, or NULL). */
mm_status mm_plan_get_config(const mm_plan *plan, int *variant, int *order_out);
/* Set them (order NULL keeps it; a Hermite plan's order cannot change).
 * Variants 0..2 as for mm_plan_autotune; 3 = every product of a
 * mumode_step call in one persistent launch of the CTA-pair kernel (F16X6
 * Tucker plans with row tiles of at most 64; other plans and calls launch
 * per product).  The autotuner does not try 3.  Drops the plan's captured
 * graphs.  Errors: MM_ERR_INVALID_ARG, MM_ERR_UNSUPPORTED. */
mm_status mm_plan_set_config(mm_plan *plan, int variant, const int *order);

/* CUDA graphs (on by default; not from the paper).  With graphs on, the
 * tensor-core paths of mumode_step, hermite_ho_step and split_step_gpe
 * capture their whole launch sequence (split, nsteps sweeps, merge) the
 * first time they are called with a given tensor pointer, nsteps, stream,
 * tau and beta, and replay that graph afterwards (at most 16 graphs per
 * plan).  Graphs are not used on the legacy default stream (NULL) or while
 * kernel timing is on.  Turning graphs off frees the cached graphs. */
mm_status mm_plan_set_graphs(mm_plan *plan, int enable);

/* Even/odd folding (not from the paper; on by default).  A direction
 * whose matrix is centrosymmetric (E_ij = E_(n-1-i, n-1-j): the
 * Dirichlet finite-difference propagators, Hermite propagators of even
 * potentials at the symmetric Gauss-Hermite nodes) acts on the folded
 * vector (x_k + x_(n-1-k) for k < n/2, then x_k - x_(n-1-k); the middle
 * entry of an odd n as it is) as a block-diagonal matrix of two half-size
 * blocks, which the tensor-core kernels run as half-size products.  With
 * folding on, the steps of a tensor-core Tucker plan (mumode_step, its
 * batches) and the harmonic-oscillator and GPE steps of an F16X6 Hermite
 * plan fold the state once per call, run on the folded state and unfold it
 * at the end (GPE: the nonlinear phase is a pass on the folded state between
 * the linear flows, unfolding, multiplying and refolding each orbit of
 * mirror points); a call folds when it is long enough for the saved tensor
 * work to pay for these passes.  The results agree with the unfolded form to
 * the precision's rounding.
 * Plans on complex64 data only; MM_NO_FOLD set (to other than 0) when a
 * plan is made turns it off for that plan.  mm_plan_get_fold reports the
 * folded directions (bit v: direction v + 1; 0: none) and
 * mm_plan_set_fold turns folding off (0) or back on; it drops the plan's
 * captured graphs.  Errors: MM_ERR_INVALID_ARG. */
mm_status mm_plan_get_fold(const mm_plan *plan, int *mask_out);
mm_status mm_plan_set_fold(mm_plan *plan, int enable);

/* Tensor-core flops (2 M N K summed over the issued MMAs) of one step of a
 * tensor-core Tucker plan: all piece products, the zero padding, and none
 * of the matrix blocks skipped because every piece of them is zero.  For
 * roofline accounting.  MM_ERR_INVALID_ARG for other plans. */
mm_status mm_plan_issued_flops(const mm_plan *plan, double *flops_per_step);

/* ---------------------------------------------------------------------
 * Batches of independent problems (not in the paper): many Tucker plans of
 * different sizes stepped together, every direction of every problem in
 * one persistent launch (the work items of all problems are dealt to the
 * same clusters of CTAs).  The plans must be tensor-core plans with the same
 * precision, d and mode order; each keeps its own matrices and workspace,
 * so a plan must not be stepped on its own while a batch step that holds
 * it is in flight.  The batch keeps device copies of the per-problem launch
 * records and refers to the plans, which must outlive it.
 * ------------------------------------------------------------------- */
typedef struct mm_batch mm_batch;
mm_status mumode_batch_create(mm_ctx *ctx, mm_plan *const *plans, int nprob, mm_batch **out);
/* nsteps steps of every problem: u_dev[k] is problem k's tensor (in place).
 * Results equal those of mumode_step on each plan. */
mm_status mumode_batch_step(mm_batch *batch, void *const *u_dev, int64_t nsteps, void *stream);
void mm_batch_destroy(mm_batch *batch);
/* The same in one call: a batch over plans[0..nprob) made, stepped nsteps
 * times with u_dev[k] in place, and released (the batch's set-up, tensor
 * maps and records, is repeated on every call; keep a batch for many
 * calls).  Errors as mumode_batch_create and mumode_batch_step. */
mm_status mumode_step_batched(mm_ctx *ctx, mm_plan *const *plans, void *const *u_dev, int nprob, int64_t nsteps,
                              void *stream);
/* Autotuner for batches: times every mode order (d <= 4) of a batch over
 * plans[0..nprob), nsteps steps each (1..1000, after one warm step), on
 * scratch copies of u_dev[k] (left unchanged), and sets the fastest order
 * on every plan; order_out (d ints, or NULL) receives it.  Allocates the
 * scratch copies for the call.  Errors: MM_ERR_INVALID_ARG, MM_ERR_OOM, and
 * those of the batch calls (the plans' order is then unchanged). */
mm_status mumode_batch_autotune(mm_ctx *ctx, mm_plan *const *plans, void *const *u_dev, int nprob, int64_t nsteps,
                                int *order_out, void *stream);

/* ---------------------------------------------------------------------
 * Hermite spectral method (section 3; section 4.3 HKP) for d = 3 with
 * m = n_mu Gauss-Hermite nodes per direction (square transforms).
 * ------------------------------------------------------------------- */

/* Plan holding the forward / backward Hermite matrices of every direction
 * and the harmonic-oscillator propagators.  dtype MM_C64 with a BF16*
 * precision or MM_PREC_FP32_SIMT, or MM_C128 with MM_PREC_FP64_SIMT. */
mm_status hermite_plan_create(mm_ctx *ctx, int d, const int64_t *n, mm_dtype dtype, mm_prec prec,
                              mm_plan **out);

/* Nodes and plain-integral weights of direction mu (1-based). */
mm_status hermite_nodes(const mm_plan *plan, int mu, double *x_out, double *W_out);

/* values at the nodes -> coefficients: F_hat = F x_1 Phi_1^W ... (eq. (real2spec)). */
mm_status hermite_forward(mm_plan *plan, const void *values_dev, void *coeffs_dev, void *stream);

/* coefficients -> values at the nodes: F = F_hat x_1 Psi_1 ... (eq. (spec2real)). */
mm_status hermite_backward(mm_plan *plan, const void *coeffs_dev, void *values_dev, void *stream);

/* nsteps exact steps of i psi_t = -1/2 Lap psi + |x|^2/2 psi (HKP with the
 * harmonic potential): forward transform, phase exp(-i tau (k1+k2+k3+3/2)),
 * backward transform.  The three factors of every direction are folded
 * into one complex matrix Psi_mu D_mu Phi_mu^W (the phase is separable),
 * so a step is three complex mu-mode products.  In place. */
mm_status hermite_ho_step(mm_plan *plan, void *psi_dev, double tau, int64_t nsteps, void *stream);

/* HKP with a potential in Kronecker form (section 4.3),
 *   i psi_t = -1/2 Lap psi + (V_1(x_1) + ... + V_d(x_d)) psi.
 *
 * mm_hermite_hamiltonian: the Hamiltonian of one direction in the m
 * Hermite functions, m x m real symmetric, row-major into H_out:
 *   H[j][k] = (k + 1/2) delta_jk + sum_l phi_j(x_l) W_l (V_l - x_l^2/2) phi_k(x_l),
 * i.e. the harmonic part -1/2 d^2/dx^2 + x^2/2 (diagonal, section 3) plus
 * the Gauss-Hermite Galerkin matrix of V - x^2/2.  V_nodes holds V at the
 * m nodes of mm_gauss_hermite(m), ascending; NULL means V = x^2/2 (H is
 * then diagonal).
 *
 * hkp_plan_create: a Tucker plan (use mumode_step, mm_plan_autotune, ...)
 * whose direction-mu matrix is the values-space propagator
 *   M_mu = Psi_mu exp(-i tau H_mu) Phi_mu^W
 * (backward transform, exact flow in coefficient space, forward transform,
 * folded into one complex n_mu x n_mu matrix in FP64; the Hamiltonian, the
 * exponential (as mm_expm_device) and the foldings run on the GPU, which
 * the call synchronises).  A step advances psi, given by its values on the
 * tensor grid of the Gauss-Hermite nodes (n[mu-1] nodes in direction mu,
 * i_1 fastest), by tau with no time-discretisation error.  V_nodes[mu-1]
 * as above (NULL,
 * or V_nodes NULL, for harmonic directions).  dtype, prec and mode_order
 * as for mumode_plan_create (complex dtypes only; tensor-core precisions
 * need n_mu <= 512).  Errors: MM_ERR_SHAPE for n_mu outside 1..4096, those
 * of mumode_plan_create. */
mm_status mm_hermite_hamiltonian(int m, const double *V_nodes, double *H_out);
mm_status hkp_plan_create(mm_ctx *ctx, int d, const int64_t *n, const double *const *V_nodes, double tau,
                          mm_dtype dtype, mm_prec prec, const int *mode_order, mm_plan **out);

/* HKMP (section 4.4): a time-dependent potential in Kronecker form,
 *   i psi_t = -1/2 Lap psi + sum_mu (V_mu(x_mu) + f(t) U_mu(x_mu)) psi,
 * Hermite pseudospectral in space and the order-two Magnus integrator
 * (eq. (mag2), exponential midpoint rule) in time.  In coefficient space
 * the midpoint operator is in Kronecker form, so a step is the Tucker
 * operator of exp(-i tau (H_mu + f_mid G_mu)), H_mu as in
 * mm_hermite_hamiltonian (from V_mu) and G_mu the Gauss-Hermite Galerkin
 * matrix of U_mu.
 *
 * hkmp_plan_create: V_nodes[mu-1] (NULL, or V_nodes NULL: harmonic) and
 * U_nodes[mu-1] (NULL, or U_nodes NULL: no time dependence in direction
 * mu) at the mm_gauss_hermite nodes.  Directions without U keep their
 * exponential, computed once on the host; those with U recompute it on the
 * GPU every step (mm_expm_device's algorithm, bound from the host 1-norms
 * of H and G) and, on the tensor cores, re-split it there.  Precisions:
 * tensor-core ones with MM_C64, or MM_PREC_FP64_SIMT / MM_PREC_FP64_DMMA
 * with MM_C128.  The plan is also a Hermite plan (hermite_forward, ...).
 *
 * hkmp_evolve: psi_dev holds the values at the nodes (i_1 fastest); the
 * call transforms them forward, takes nsteps Magnus steps of the plan's
 * tau in coefficient space with f_mid[k] = f(t_k + tau/2) (host array of
 * nsteps doubles), and transforms back, in place.  The fixed-point state
 * and the coefficients stay on the device between steps.  Since every
 * f_mid is known at the call, the exponentials of up to 64 steps are
 * computed together (batched real products, see mm_expm_device).  On
 * tensor-core plans the series is scaled to norm 2 (truncation below
 * 5e-13), and a chunk of more than K steps takes its exponentials from
 * K Chebyshev nodes in f over the chunk's f range (K = 4..12, the fewest
 * whose interpolation error bound 2 (tau ||G||_1 (f_hi - f_lo) / 4)^K / K!
 * is below 1e-14), both below the resolution of the tensor-core pieces;
 * FP64 plans compute every step's exponential to full FP64 accuracy.  The
 * call synchronises the stream before returning (f_mid is then no longer
 * read). */
mm_status hkmp_plan_create(mm_ctx *ctx, int d, const int64_t *n, const double *const *V_nodes,
                           const double *const *U_nodes, double tau, mm_dtype dtype, mm_prec prec, mm_plan **out);
mm_status hkmp_evolve(mm_plan *plan, void *psi_dev, int64_t nsteps, const double *f_mid, void *stream);

/* Declares a range [f_lo, f_hi] that f_mid takes (not from the paper; for
 * f = sin^2 t, [0, 1]).  The plan computes the exponentials at the K
 * Chebyshev nodes of that range once (K = 4..12 by the bound above, on
 * stream, which is synchronised) and keeps them; from then on every chunk
 * of hkmp_evolve whose f values all lie in the range combines its steps'
 * exponentials from those nodes instead of computing nodes of its own
 * (chunks with a value outside it do as before).  The interpolation error
 * stays below 1e-14, under the pieces' resolution.  f_lo >= f_hi drops a
 * declared range.  Errors: MM_ERR_INVALID_ARG (not an HKMP plan, a bound
 * not finite, a range needing more than 12 nodes), MM_ERR_UNSUPPORTED (an
 * FP64 plan: its steps take exact exponentials), MM_ERR_OOM (12 matrices
 * per time-dependent direction), MM_ERR_CUDA. */
mm_status hkmp_set_f_range(mm_plan *plan, double f_lo, double f_hi, void *stream);

/* nsteps Strang steps of i psi_t = -1/2 Lap psi + |x|^2/2 psi + beta |psi|^2 psi
 * (section 4.5): half linear step, exact nonlinear phase
 * psi <- psi exp(-i tau beta |psi|^2), half linear step.  Adjacent linear
 * halves of consecutive steps are merged into one full step; the nonlinear
 * phase is applied in the epilogue of the last mode product.  In place. */
mm_status split_step_gpe(mm_plan *plan, void *psi_dev, double beta, double tau, int64_t nsteps,
                         void *stream);

/* split_step_gpe, then the weighted norm sum_x |psi(x)|^2 W1(x1) W2(x2) W3(x3)
 * of the result (the Gauss-Hermite quadrature of ||psi||^2, the conserved
 * mass of section 4.5) in FP64 to *norm2_host (host memory); the stream is
 * synchronised.  On F16X6 plans with the CTA-pair kernel the sum is taken in
 * the epilogue of the last mode product, from the FP32 values before they
 * are split (one FP64 atomic per epilogue warp), or, when the steps run on
 * the even/odd-folded state, by the pass that unfolds the result (from the
 * complex64 values it writes), so no pass re-reads psi; otherwise the steps
 * are followed by mm_norm2(weighted).  nsteps = 0 gives
 * the norm of psi_dev.  3D Hermite plans only.  Errors: those of
 * split_step_gpe and mm_norm2, MM_ERR_INVALID_ARG (not a 3D Hermite plan,
 * norm2_host NULL), MM_ERR_OOM (the plan's 8-byte accumulator). */
mm_status split_step_gpe_norm2(mm_plan *plan, void *psi_dev, double beta, double tau, int64_t nsteps,
                               double *norm2_host, void *stream);

/* Gradient of a real loss J(psi_T), psi_T = nsteps Strang steps of psi0
 * (split_step_gpe with the same beta, tau), with respect to psi0 (reverse
 * mode; not in the paper).  Gradients are g = dJ/dRe psi + i dJ/dIm psi, so
 * that dJ = Re <g, delta> (the convention of torch autograd for complex
 * tensors).  gT_dev holds the gradient at psi_T, g0_dev receives the one at
 * psi0 (g0 may alias gT, not psi0).  The linear flows enter through their
 * conjugate transposes (mu-mode products with Psi D(s) Phi_W transposed
 * and conjugated); the nonlinear stage psi' = psi e^{-i theta},
 * theta = tau beta |psi|^2, through g = e^{i theta} g' + 2 tau beta
 * Im(conj(g') psi') psi.  Forward states are kept every ckpt_every steps
 * and recomputed within a segment (memory: ceil(nsteps / ckpt_every) +
 * ckpt_every + 1 states).  The first call builds the propagators of the
 * forward and adjoint half and full steps and allocates the checkpoint
 * buffers; both stay with the plan (buffers grow when a later call needs
 * more, matrices are rebuilt when tau changes) until mm_plan_destroy.
 * Calls on one plan must not overlap.  The call synchronises the stream. */
mm_status split_step_gpe_adjoint(mm_plan *plan, const void *psi0_dev, const void *gT_dev, void *g0_dev,
                                 double beta, double tau, int64_t nsteps, int64_t ckpt_every,
                                 void *stream);

/* The autotuner (mm_plan_autotune) timing GPE steps with this beta and tau
 * instead of harmonic-oscillator steps: the nonlinear epilogue changes
 * which kernel variant is fastest.  Same arguments and errors otherwise. */
mm_status split_step_gpe_autotune(mm_plan *plan, const void *psi_dev, double beta, double tau, int64_t nsteps,
                                  void *stream);

/* FP64 sum of |u|^2 (times w_l = W_l1 W_l2 W_l3 for a Hermite plan when
 * weighted != 0) over the plan's tensor; the result is written to
 * *out_host after synchronising the stream.  The weighted sum of complex64
 * data squares each value in FP32 (an unbiased rounding, 1e-10 or so on
 * the sum) and multiplies by the FP64 weight: one FP64 operation a point. */
mm_status mm_norm2(mm_plan *plan, const void *u_dev, int weighted, double *out_host, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* MUMODE_H */
