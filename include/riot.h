/*
 * riot.h -- C ABI of a single-GPU (GB300, sm_103a) library for the inner loop
 * of RIOT, the Randomized Incremental Optimal Technique for incremental
 * 4D-Var (Bousserez, Guerrette & Henze, arXiv:1906.01413).
 *
 * The library owns one assimilation window per context.  Each outer
 * iteration integrates the nonlinear model and forms the gradient
 * (riot_outer_begin); the inner loop is a randomized eigendecomposition of
 * the prior-preconditioned Hessian A = L^T H^T R^-1 H L built from batched
 * tangent-linear + adjoint integrations (riot_hessian_apply, riot_rsvd),
 * followed by the adaptive low-rank increment (riot_increment) and the
 * low-rank analysis covariance (riot_analysis_cov_lowrank).
 *
 * Conventions shared by every entry point
 *  - Arguments named *_dev are device pointers on the context's device,
 *    owned by the caller; the library never frees them.  Host arrays are
 *    read during the call only.
 *  - Vectors of length n are contiguous.  Blocks of column vectors are
 *    column-major: column j of an n x m block starts at ptr + j*ld.
 *  - Element type of the Hessian blocks (W, Y, Omega): float when the
 *    context was created with RIOT_PREC_MIXED, double with RIOT_PREC_FP64.
 *    Outer-loop vectors (x, v, dv, U, L U) are always double.
 *  - Work is queued on the stream given to riot_setup.  Calls that return
 *    host scalars (J, eigenvalues, mode) synchronise that stream; the
 *    others are asynchronous.
 *  - Calls never throw; they return a riot_status.  riot_last_error gives a
 *    one-line message for the last failing call on the context.  Calls made
 *    out of order (e.g. riot_increment before riot_rsvd) return RIOT_ESTATE.
 *  - Sign conventions follow Algorithm 3: d = H(x) - y, dv = -(...)(b + v).
 *    Eigenvalues are those of A (not I + A), sorted in decreasing order.
 *  - One context is not safe to use from two host threads at once.
 *  - Kernels with bounded device waits (the mixed-precision Hessian kernel's
 *    stage copies, the tensor-core GEMMs) never hang: a wait that runs out
 *    raises a flag and the kernel finishes with invalid results.  Every call
 *    that launches such kernels clears the flag when it starts and reads it
 *    before it returns (this synchronises), returning RIOT_ETIMEOUT; the
 *    context stays usable and the next call starts clean.
 */
#ifndef RIOT_H
#define RIOT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    RIOT_OK = 0,
    RIOT_EINVAL = -1,    /* bad argument or descriptor                        */
    RIOT_ENOMEM = -2,    /* device allocation failed                          */
    RIOT_ECUDA = -3,     /* a CUDA runtime call failed                        */
    RIOT_ENOTSPD = -4,   /* Cholesky met a non-positive pivot (no fallback)   */
    RIOT_ETIMEOUT = -5,  /* a bounded device wait ran out                     */
    RIOT_ESTATE = -6,    /* call out of order                                 */
    RIOT_ENOCONV = -7,   /* the eigensolver did not converge                  */
    RIOT_ENONFINITE = -8 /* a NaN or Inf reached a reduction                  */
} riot_status;

enum { RIOT_MODEL_L96 = 1, RIOT_MODEL_ADVDIFF = 2 };
enum { RIOT_B_GAUSS_RING = 1, RIOT_B_EXP_SEPARABLE = 2 };
enum { RIOT_PREC_MIXED = 0, RIOT_PREC_FP64 = 1 };
enum { RIOT_EIG_TRIDIAG = 0, RIOT_EIG_JACOBI = 1 };

/* Tracer transport for a surface-emission inversion (the setting of the
 * paper's black-carbon experiments, Section 3.2, on a synthetic box model).
 * Cells (i, j, l), i < nx periodic in x, j < ny between solid walls, l < nz
 * levels with zero flux at the bottom and top; cell (i, j, l) is centred at
 * (i, j, l) in cell units.  dc/dt = A c + s with
 *  - upwind flux-form advection by the steady face winds amp[l] * u (x-face
 *    i-1/2 of row j, u[j*nx + i]) and amp[l] * v (y-face j-1/2 of column i,
 *    v[j*nx + i], j = 0..ny; rows 0 and ny are the walls and must be 0);
 *  - vertical diffusion with diffusivity kz[l] on face l-1/2 (l = 1..nz-1;
 *    kz[0] and kz[nz] are ignored: no flux through the bottom and top);
 *  - the surface source s = E / dz in level 0, E = emis_b * exp(x) where the
 *    control x holds one value per surface cell and emission block:
 *    x[(b*ny + j)*nx + i], n = nblocks*ny*nx.  Step t (0-based) uses block
 *    t*nblocks/T.  The tracer starts at 0.
 * Time stepping is classical RK4 with s held over each step.  All arrays are
 * host arrays read during riot_setup.  Limits: nx >= 2, 2 <= ny, 2 <= nz <= 32,
 * 1 <= nblocks <= T, amp > 0, kz >= 0, emis_b finite. */
typedef struct {
    int32_t nx, ny, nz, nblocks;
    double dx, dy, dz;          /* cell sizes (m)                                 */
    const double *u;            /* [ny][nx]   x-face velocities (m/s)             */
    const double *v;            /* [ny+1][nx] y-face velocities (m/s)             */
    const double *amp;          /* [nz]       level scaling of u and v            */
    const double *kz;           /* [nz+1]     face diffusivities (m^2/s)          */
    const double *emis_b;       /* [nblocks][ny][nx] background emissions         */
} riot_advdiff_desc;

/* Model of the window.
 * RIOT_MODEL_L96 (Section 3.1): dx_i/dt = (x_{i+1} - x_{i-2}) x_{i-1} - x_i + F
 * on a periodic ring of n variables, advanced by T classical RK4 steps of
 * length dt.  Limits: 16 <= n <= 8192, 0 <= T, dt > 0.  advdiff is ignored.
 * RIOT_MODEL_ADVDIFF: the tracer model of riot_advdiff_desc (required);
 * n must equal nblocks*ny*nx, T >= 1 steps of length dt; F is ignored. */
typedef struct {
    int32_t kind;   /* RIOT_MODEL_L96 or RIOT_MODEL_ADVDIFF                   */
    int32_t T;      /* number of time steps in the window                     */
    int64_t n;      /* control size                                           */
    double dt;      /* step length                                            */
    double F;       /* forcing (Lorenz-96)                                    */
    const riot_advdiff_desc *advdiff;   /* RIOT_MODEL_ADVDIFF only            */
} riot_model_desc;

/* Observations y with diagonal error covariance R = diag(sigma^2)
 * (Section 2.1, Eq. 2), each taken at the end of step step[j] (step 0 = the
 * initial state).  Entries must be sorted by step (nondecreasing).
 * Lorenz-96: observation j is of variable idx[j]; several observations of
 * one (step, idx) pair are allowed; pos is ignored.
 * Tracer model: observation j is the trilinear interpolation of the tracer
 * at pos[3j..3j+2] = (x, y, z) in cell units (x periodic, any real; y in
 * [0, ny-1]; z in [0, nz-1]); idx is ignored; step >= 1.
 * All arrays are host arrays of length p (pos: 3p); p = 0 is allowed. */
typedef struct {
    int64_t p;
    const int32_t *step;   /* 0..T                          */
    const int32_t *idx;    /* 0..n-1 (Lorenz-96)            */
    const double *y;       /* observed value                */
    const double *sigma;   /* error standard deviation > 0  */
    const double *pos;     /* 3p cell coordinates (tracer)  */
} riot_obs_desc;

/* Prior covariance B = L L^T (Section 2.1, Eq. 3).
 * RIOT_B_EXP_SEPARABLE (tracer model only): L = sigma_b (S_y kron S_x) on
 * each emission block, blocks independent, with S_x, S_y the symmetric
 * square roots (eigenvalues below 0 set to 0) of the exponential
 * correlations exp(-d / length), d the periodic x distance (times dx) and
 * the y distance (times dy); sigma_vec must be NULL.
 * RIOT_B_GAUSS_RING (Lorenz-96, the Gaussian correlations of Section 3.1):
 * L = diag(s) S with S the periodic
 * Gaussian convolution S_d = alpha sum_j exp(-(d + j n)^2 / length^2),
 * normalised so that (S S^T)_ii = 1.  Then B = L L^T has the Gaussian
 * correlation exp(-d^2 / (2 length^2)) up to lattice terms of relative size
 * 2 exp(-pi^2 length^2 / 2).  S is applied as a band of the offsets whose
 * weight exceeds 1e-18 of the peak.
 * s = sigma_vec (host, length n) when non-NULL, else sigma_b everywhere. */
typedef struct {
    int32_t kind;
    int32_t reserved;
    double length;
    double sigma_b;
    const double *sigma_vec;
} riot_bcov_desc;

/* Caller-supplied device allocator (riot_options.dev_alloc / dev_free), so that a
 * host framework's caching allocator serves the context's workspace.  dev_alloc
 * returns `bytes` of device memory on the current device, aligned to at least 256
 * bytes, usable in stream order on cuda_stream (the context's stream), or NULL;
 * dev_free gives back a pointer dev_alloc returned, with the same size and stream.
 * Both are called from the thread that calls riot_setup, riot_precond_enable,
 * riot_psas (first call) and riot_destroy, and only there. */
typedef void *(*riot_dev_alloc_fn)(size_t bytes, void *cuda_stream, void *user);
typedef void (*riot_dev_free_fn)(void *ptr, size_t bytes, void *cuda_stream, void *user);

typedef struct {
    int32_t precision;  /* RIOT_PREC_MIXED: FP32 TL/AD and FP32 block storage,
                           FP64 Gram/Cholesky, eigensolver and increment;
                           RIOT_PREC_FP64: double everywhere                  */
    int32_t kmax;       /* largest number of sketch columns used per call (>= 1) */
    int32_t exact_rr;   /* 0: K solves K (Q^T W) = Q^T Y (Algorithm 3);
                           1: K = Q^T A Q (k more Hessian applications)       */
    int32_t eig_method; /* k x k eigensolver, FP64: RIOT_EIG_TRIDIAG (Householder
                           tridiagonalisation + bisection + inverse iteration,
                           default) or RIOT_EIG_JACOBI (parallel cyclic Jacobi) */
    uint64_t seed;      /* key of the device-drawn Gaussian sketch            */
    riot_dev_alloc_fn dev_alloc; /* NULL (with dev_free NULL): cudaMalloc / cudaFree */
    riot_dev_free_fn dev_free;   /* given together with dev_alloc                 */
    void *alloc_user;            /* passed through to dev_alloc / dev_free        */
} riot_options;

typedef struct riot_ctx riot_ctx;

/* Create a context on the current CUDA device.  Copies the model, the
 * observations and the B descriptor to the device, builds L, and allocates
 * all workspace for kmax sketch columns (through opt->dev_alloc when given;
 * a NULL from it is RIOT_ENOMEM, a pointer not aligned to 256 bytes
 * RIOT_EINVAL).  It also looks up, once per device, the device address of
 * the static scratch array of riot_hessian_apply_noalloc.  cuda_stream is a
 * cudaStream_t (NULL = legacy default stream).  On failure *out is NULL. */
riot_status riot_setup(riot_ctx **out, const riot_model_desc *model, const riot_obs_desc *obs,
                       const riot_bcov_desc *B, const riot_options *opt, void *cuda_stream);

/* Outer-loop prerequisites (Algorithm 3, top of the outer loop): set the
 * current state x (and control-space increment sum v, NULL = 0 on the first
 * call, else the context's own v), integrate and store the trajectory in
 * FP64, form d = H(x) - y, the cost J = 1/2 ||R^-1/2 d||^2 + 1/2 ||v||^2,
 * the gradient b = L^T H^T R^-1 d (one FP64 adjoint integration) and
 * g = b + v.  x_dev NULL keeps the context's x (updated by riot_increment).
 * J_out (host, may be NULL) receives J; this synchronises. */
riot_status riot_outer_begin(riot_ctx *ctx, const double *x_dev, const double *v_dev, double *J_out);

/* Y = A W (+ W when add_identity), A = L^T sum_t M_{0->t}^T H_t^T R^-1 H_t
 * M_{0->t} L (Eq. 4): for every column, one tangent-linear integration
 * forward and one adjoint integration backward along the stored trajectory
 * (Algorithm 3, "do in parallel").  W and Y are n x ncols blocks with
 * leading dimension ld >= n (element type per the precision).  ncols may
 * exceed kmax (processed in slices).  Requires riot_outer_begin. */
riot_status riot_hessian_apply(riot_ctx *ctx, const void *W_dev, void *Y_dev, int64_t ld,
                               int32_t ncols, int32_t add_identity);

/* Same result as riot_hessian_apply, for callers that must not allocate
 * device memory when they apply the Hessian: for example code that runs
 * under a memory pool or budget that forbids cudaMalloc after start-up, or
 * a context created with a small kmax whose residual workspace is too small
 * for the block at hand.  (The paper has no counterpart: this is a property
 * of the library, not of the method.)  The tangent-linear residuals that
 * wait for the adjoint pass go to a fixed 16 MiB device array inside the
 * library instead of the context's workspace; the columns are processed in
 * slices that fit it, so any ncols is accepted.  If one column alone needs
 * more than 16 MiB (p observations x 4 bytes in RIOT_PREC_MIXED, x 8 bytes in
 * RIOT_PREC_FP64) the call returns RIOT_EINVAL and does nothing.
 *  - Nothing is allocated: no cudaMalloc, cudaFree or allocating library call.
 *  - The array belongs to the process, one copy per device that loaded the
 *    library, held until exit.  Its device address is looked up once per
 *    device by riot_setup, so this entry point itself does no lookup.
 *  - All calls share the array and it keeps the last call's contents.  Each
 *    call writes every residual it reads, so nothing needs clearing, but two
 *    calls that overlap on the GPU (other streams, other contexts on the same
 *    device) race on it.
 * Arguments, layout and errors are those of riot_hessian_apply. */
riot_status riot_hessian_apply_noalloc(riot_ctx *ctx, const void *W_dev, void *Y_dev, int64_t ld,
                                       int32_t ncols, int32_t add_identity);

/* Randomized eigendecomposition of A (Algorithm 3 inner loop): draw Omega
 * (n x k, N(0,1)) from the context seed and sketch_stream with Philox4x32-10
 * + Box-Muller unless Omega_dev (n x k, ld = n) is given; Y = A Omega; q
 * rounds of subspace iteration Q = orth(Y), Y = A Q; Q = orth(Y) by shifted
 * CholeskyQR with two cleanup passes; K from Q^T W and Q^T Y (or Q^T A Q);
 * K = Z Lambda Z^T in FP64 (options.eig_method); U = Q Z.  1 <= k <= min(kmax, n).
 * lambda_out (host, k doubles, may be NULL) receives the eigenvalues in
 * decreasing order; this synchronises.  Requires riot_outer_begin. */
riot_status riot_rsvd(riot_ctx *ctx, int32_t k, int32_t q, int64_t sketch_stream,
                      const void *Omega_dev, double *lambda_out);

/* Deflated multi-level randomized eigendecomposition for mixed-precision
 * contexts (an extension of Algorithm 3 for FP32 Hessian products; the paper
 * has no counterpart).  An FP32 product carries an absolute error of about
 * 2^-24 lambda_1 |w|, so riot_rsvd in RIOT_PREC_MIXED resolves only the pairs
 * above that; on strongly unstable windows the rest of the spectrum carries
 * much of the cost reduction.  That error lies almost entirely in the leading
 * eigen-directions, so projecting them out recovers the next part of the
 * spectrum.  Level l = 0 .. nlevels-1 runs Algorithm 3 (q power iterations)
 * with min(kcols[l], kmax - m, n - m) columns of a sketch of its own (Philox
 * stream sketch_stream with its top four bits replaced by l) on the deflated
 * operator P A P, P = I - U U^T with U the m pairs kept by the levels before
 * (P = I at level 0); every block is projected by P, in two passes of FP32
 * tensor-core GEMMs, before and after each FP32 Hessian product.  A level
 * keeps its leading pairs with lambda >= rel_floor times its largest one
 * (rel_floor <= 0: 2^-24, the absolute error of its FP32 products of unit
 * vectors) and, after level 0, above 1.  The levels stop early when one's
 * largest eigenvalue is below 1 or below 2^-53 lambda_1 (unresolved even by
 * FP64 products).  The m pairs of all levels, sorted by decreasing
 * eigenvalue, become the context's pairs for riot_increment and
 * riot_analysis_cov_lowrank (all m are retained).  lambda_out (host, room for
 * kmax doubles, may be NULL) and m_out (may be NULL) receive them;
 * synchronises.  1 <= nlevels <= 8; 1 <= kcols[0] <= min(kmax, n); later
 * kcols in [0, kmax].  Requires riot_outer_begin and a RIOT_PREC_MIXED
 * context without spectral preconditioner.
 * Measured on 4096-variable, 200-step windows (spectra over twelve to
 * thirteen decades): two levels ({256, 320}) reach 0.93 to 1.01 of the cost
 * reduction of the FP64 rank-512 increment; deeper levels reach eigenvalues
 * whose FP32 Ritz vectors are no longer accurate (the part of the products'
 * error outside the kept subspace is then of their size) and the increment's
 * cost rises, so two levels are the depth to use. */
riot_status riot_rsvd_deflated(riot_ctx *ctx, int32_t nlevels, const int32_t *kcols, int32_t q, double rel_floor,
                               int64_t sketch_stream, double *lambda_out, int32_t *m_out);

/* Adaptive increment (Algorithm 3, Eqs. 8-11): with c = U^T g over the
 * retained pairs,
 * LRA (mode 0) when the smallest retained eigenvalue is > 1:
 *     dv = -U diag(1/(1+lambda)) c
 * LRU (mode 1) otherwise:  dv = -(g - U diag(lambda/(1+lambda)) c).
 * RIOT_PREC_FP64 retains all k pairs of riot_rsvd.  RIOT_PREC_MIXED retains
 * the leading pairs with lambda >= 2^-24 lambda_1: an FP32 Hessian product
 * carries an absolute error of about 2^-24 lambda_1 |w| (its rounding, carried
 * along the window's leading growth), so smaller Ritz values are not
 * determined by the products and would decide the mode at random.
 * Then v += dv and x += L dv in the context.  dv_dev (n doubles) and
 * mode_out may be NULL; a non-NULL mode_out synchronises.  Requires
 * riot_rsvd since the last riot_outer_begin.  The stored trajectory and g
 * are those of the last riot_outer_begin until the next one, so repeated
 * riot_rsvd / riot_increment calls redo the same inner loop. */
riot_status riot_increment(riot_ctx *ctx, double *dv_dev, int32_t *mode_out);

/* Low-rank analysis covariance (Eqs. 8/9 with B = L L^T):
 * LRU: P_a = B - (LU) diag(coef) (LU)^T, coef = lambda/(1+lambda)
 * LRA: P_a = (LU) diag(coef) (LU)^T,     coef = 1/(1+lambda)
 * for the leading m <= k eigenpairs.  LU_dev: n x m doubles (ld = n);
 * coef_out: host m doubles (may be NULL; synchronises); mode by the same
 * rule as riot_increment applied to the m retained eigenvalues. */
riot_status riot_analysis_cov_lowrank(riot_ctx *ctx, int32_t m, double *LU_dev, double *coef_out,
                                      int32_t *mode_out);

/* out = L in (transpose = 0) or L^T in (transpose = 1) for ncols columns of
 * n doubles (ld = n). */
riot_status riot_bsqrt_apply(riot_ctx *ctx, const double *in_dev, double *out_dev, int32_t transpose,
                             int32_t ncols);

/* The innovation d = H(x) - y of the last riot_outer_begin (p doubles,
 * device).  With y = 0 this is the model-equivalent H(x) of the observations,
 * which is how synthetic observations are made from a truth. */
riot_status riot_get_innovation(riot_ctx *ctx, double *d_dev);

/* Copy the context's state out: x, v, g (n doubles each), the eigenvectors
 * U (n x k doubles) and eigenvalues (k doubles, device); NULL skips one. */
riot_status riot_get_state(riot_ctx *ctx, double *x_dev, double *v_dev, double *g_dev,
                           double *U_dev, double *lambda_dev);

/* Gaussian block from the Philox4x32-10 + Box-Muller stream (seed, stream):
 * element (i, j) of the n x ncols block is stream element j*n + i, written
 * at out[j*ld + i] as float (is_double = 0) or double. */
riot_status riot_draw_normal(uint64_t seed, int64_t stream, int64_t n, int32_t ncols, int64_t ld,
                             int32_t is_double, void *out_dev, void *cuda_stream);

/* Standalone FP64 Lorenz-96 forecast: traj_dev ((T+1) x n doubles) gets the
 * RK4 trajectory from x0_dev, or only the final state when
 * store_all = 0 (traj_dev then holds n doubles).  Used to build synthetic
 * truths without a context. */
riot_status riot_l96_forecast(int64_t n, int32_t T, double dt, double F, const double *x0_dev,
                              double *traj_dev, int32_t store_all, void *cuda_stream);

/* The k x k symmetric eigensolver of riot_rsvd on its own (Algorithm 3,
 * K = Z Lambda Z^T, FP64): K_dev (k x k, column-major, read only),
 * lambda_dev (k, decreasing), Z_dev (k x k eigenvectors).  method is
 * RIOT_EIG_TRIDIAG or RIOT_EIG_JACOBI.  Allocates and frees its own
 * workspace; synchronises the stream.  1 <= k <= 4096. */
riot_status riot_symm_eig(const double *K_dev, int32_t k, double *lambda_dev, double *Z_dev, int32_t method,
                          void *cuda_stream);

/* Timings of the phases of the last riot_rsvd in milliseconds (CUDA events on
 * the context stream): [0] Hessian applications, [1] orthonormalisation,
 * [2] projected matrix K, [3] eigensolver, [4] Ritz vectors, [5] total.
 * Synchronises. */
riot_status riot_rsvd_timings(riot_ctx *ctx, double *ms_out6);

/* Launch shape of the mixed-precision Hessian kernel: sketch columns per CTA
 * and depth of its shared-memory ring(s) of streamed stage coefficients
 * (2..8); 0 = automatic.  A shape that does not fit the device falls back to
 * the automatic choice.  Used by the autotuner; results do not depend on it. */
riot_status riot_set_hvp_config(riot_ctx *ctx, int32_t probes_per_cta, int32_t ring_depth);

/* Which FP32 Hessian kernel a mixed-precision Lorenz-96 context uses (both
 * compute Eq. 4 in FP32 with the same stage coefficients, in different
 * rounding order):
 *  RIOT_HVP_CTA_BARRIER (default): the CTA streams the stage coefficients
 *    through one shared ring (1-D TMA) and exchanges chunk halos in shared
 *    memory behind one CTA-wide barrier per RK4 stage;
 *  RIOT_HVP_WARP_PAIRS: every warp streams its own chunks' coefficients
 *    through its own ring, and meets only its two neighbouring warps, at a
 *    hardware named barrier per pair, after the elements that need no other
 *    thread's values (windows with 8 or 16 variables per thread and 64 to 512
 *    threads per column; others keep the default);
 *  RIOT_HVP_WARP_SHUFFLE: RIOT_HVP_WARP_PAIRS with the halo passed by warp
 *    shuffles between the lanes of a warp, only the two edge lanes of each
 *    warp going through shared memory;
 *  RIOT_HVP_CTA_TWO_PER_SM: the default kernel with one probe per thread
 *    (64 registers) and two CTAs per SM (windows with 8 variables per thread;
 *    others keep the default).
 * The two warp kernels give the same products bit for bit.  Measured on the
 * 4096-variable, 200-step window (512 products per launch): 2.7 ms for the
 * default, 3.0 ms with warp pairs, 3.4 ms with shuffles, 3.4 ms with two CTAs
 * per SM (each CTA streams the whole coefficient stream for half the probes,
 * through a ring of two slots; the per-warp ring
 * bookkeeping costs more instructions than the CTA barrier costs waiting,
 * and the shuffles issue as many instructions as the shared-memory halo they
 * replace while lengthening the path to the barrier). */
enum { RIOT_HVP_CTA_BARRIER = 0, RIOT_HVP_WARP_PAIRS = 1, RIOT_HVP_WARP_SHUFFLE = 2, RIOT_HVP_CTA_TWO_PER_SM = 3 };
riot_status riot_set_hvp_kernel(riot_ctx *ctx, int32_t kernel);

/* Bound of every wait of the mixed-precision Hessian kernels (on a stage copy,
 * or on a neighbouring warp's edge values), in tries of the waited mbarrier:
 * polls >= 0 sets it (0 gives up at once, so the next Hessian application
 * reports RIOT_ETIMEOUT without a fault: this is how the timeout report is
 * tested), polls < 0 restores the default (a wait gives up after well under a
 * second).  Whatever the bound, a kernel whose wait ran out still waits with
 * the default bound for every copy it started before its blocks exit. */
riot_status riot_set_wait_limit(riot_ctx *ctx, int32_t polls);

/* Inner-loop quadratic cost (Eq. 3 with Algorithm 3's sign of d)
 *     J~(dv) = 1/2 ||R^-1/2 (d + H M L dv)||^2 + 1/2 ||v + dv||^2
 * at the linearisation of the last riot_outer_begin (its trajectory, d and
 * v), in FP64 on either precision: one FP64 tangent-linear integration of
 * L dv.  dv_dev: n doubles (NULL: J~(0), the cost J of riot_outer_begin).
 * The cost reduction of an increment is J~(0) - J~(dv).  *J_out (host) gets
 * the value; this synchronises.  Requires riot_outer_begin. */
riot_status riot_quadratic_cost(riot_ctx *ctx, const double *dv_dev, double *J_out);

/* Number of eigenpairs the last increment retained (m <= k, see
 * riot_increment; after riot_increment or a batch inner loop).  Synchronises. */
riot_status riot_increment_pairs(riot_ctx *ctx, int32_t *m_out);

/* Number of Jacobi sweeps of the last successful riot_rsvd (-1: no context). */
int32_t riot_rsvd_sweeps(const riot_ctx *ctx);

/* Number of kernel launches the library has issued in this process (all
 * contexts); a benchmark reads it before and after a timed region. */
uint64_t riot_kernel_launches(void);

/* Measured arithmetic peaks of GPU `device` (a measurement utility for the
 * roofline fractions of the ALU-bound kernels, not part of the method):
 *   out[0] FP64 FMA throughput, TFLOP/s (eight independent FMA chains per
 *          thread, four CTAs of 256 threads per SM, best of three launches
 *          timed with CUDA events after one warm-up);
 *   out[1] FP32 FMA throughput, TFLOP/s (the same kernel in FP32);
 *   out[2] FP64 FMA latency, SM cycles per dependent FMA (one thread);
 *   out[3] FP64 rsqrt latency, SM cycles per dependent rsqrt + add;
 *   out[4] FP64 division latency, SM cycles per dependent division + add;
 *   out[5] latency of the refined reciprocal the FP64 k x k chains use (the
 *          hardware approximation plus one third-order Newton step), SM
 *          cycles per dependent reciprocal + add;
 *   out[6] its largest error, in ulps of the correctly rounded reciprocal,
 *          over 2^24 inputs of both signs log-uniform in [2^-1100, 2^1100]
 *          and the range limits.
 * Writes min(nout, 7) values.  Runs on its own stream, allocates about
 * 2 MB for the run, synchronises; takes about 40 ms.  RIOT_EINVAL for a null
 * out or nout < 1, RIOT_ECUDA for a CUDA error. */
riot_status riot_measure_peaks(int32_t device, double *out, int32_t nout);

/* ---- Batches of windows ------------------------------------------------------
 * Many independent Lorenz-96 windows (contexts of any n, T, observations and
 * k) run their inner loops together: the Hessian products of all windows in
 * one persistent launch per Hessian application (a queue of (window, block)
 * items over all SMs), the per-window linear algebra on parallel branches,
 * and the whole inner loop captured once as a CUDA graph and replayed.  The
 * paper runs its samples as independent jobs (Algorithm 3, "do in
 * parallel"); this extends the same independence across windows.
 * Contexts must be RIOT_PREC_MIXED, RIOT_MODEL_L96, on one device, each used
 * by one batch at a time and not otherwise while the batch runs. */
typedef struct riot_batch riot_batch;

/* Create a batch of nwin windows: window w uses ctxs[w] with k[w] sketch
 * columns (1 <= k[w] <= min(kmax, n)) and q power iterations.  The batch
 * owns one stream per window; cuda_stream is the stream its work joins.
 * The contexts are not copied: they must outlive the batch. */
riot_status riot_batch_create(riot_batch **out, riot_ctx *const *ctxs, int32_t nwin, const int32_t *k, int32_t q,
                              void *cuda_stream);

/* Time the persistent Hessian launch for a set of launch shapes (probe
 * groups per CTA capped at 0 = as many as fit, 32, 16, 8, 4, 2; ring depths
 * 4, 3, 2), keep the fastest and report it (outputs may be NULL).  Writes
 * Gaussian blocks into the windows' workspaces; requires riot_outer_begin on
 * every window.  Results never depend on the shape. */
riot_status riot_batch_autotune(riot_batch *b, int32_t *probes_cap_out, int32_t *ring_depth_out, double *ms_out);

/* Set the launch shape directly (0 = automatic); drops a captured graph. */
riot_status riot_batch_set_config(riot_batch *b, int32_t probes_cap, int32_t ring_depth);

/* Y = A W for every window in one launch, W and Y being each context's
 * internal sketch blocks (for timing and tests). */
riot_status riot_batch_hessian_apply(riot_batch *b);

/* One inner loop of every window: riot_rsvd (sketch from the window's seed
 * and sketch_stream) followed by riot_increment, as one CUDA graph
 * (use_graph = 1; captured on the first call and replayed while
 * sketch_stream stays the same) or as plain stream work (use_graph = 0).
 * Synchronises.  status_out (nwin, may be NULL) receives each window's
 * status; the return value is the first failure.  Afterwards each context
 * holds its eigenpairs and increment as after riot_rsvd + riot_increment
 * (do not call riot_increment again for the same inner loop). */
riot_status riot_batch_run(riot_batch *b, int64_t sketch_stream, int32_t use_graph, int32_t *status_out);

const char *riot_batch_last_error(const riot_batch *b);
void riot_batch_destroy(riot_batch *b);

/* ---- Learned sketch proposal ----------------------------------------------
 * A periodic 1-D convolutional network maps C_in standardised snapshots of a
 * Lorenz-96 background trajectory to m proposed sketch directions; it is
 * trained on leading Hessian eigenvectors that RIOT produced for other
 * windows.  This extends the randomized range finder of Section 2.2; the
 * Gaussian sketch of Algorithm 3 remains the fallback that decides
 * (riot_rsvd_proposal).  Network: depth periodic conv layers of width ksize
 * (odd, <= 7), tanh on the hidden layers, channels c_in -> width -> ... ->
 * m_out.  Parameters are one FP32 vector: per layer W[C_out][C_in][ksize]
 * then b[C_out].  conv(x)[o][i] = b[o] + sum_c sum_d W[o][c][d]
 * x[c][(i + d - ksize/2) mod n].  Loss per window with target U (n x r,
 * orthonormal columns) on the directions X (n x m):
 *   ||X - U U^T X||_F^2 / ||X||_F^2 + mu ||X^T X / s - I||_F^2 / m^2,
 *   s = ||X||_F^2 / m,
 * averaged over the batch; training uses Adam (beta 0.9 / 0.999, eps 1e-8). */
typedef struct riot_sketchnet riot_sketchnet;

/* Create a network with zero parameters (set them with riot_sketchnet_set_params)
 * for inputs of up to n_max variables, batches of up to batch_max windows and
 * targets of up to r_max vectors. */
riot_status riot_sketchnet_create(riot_sketchnet **out, int32_t c_in, int32_t width, int32_t m_out, int32_t depth,
                                  int32_t ksize, int32_t n_max, int32_t batch_max, int32_t r_max, void *cuda_stream);
int64_t riot_sketchnet_num_params(const riot_sketchnet *net);
/* Copy the parameters in (and restart the optimiser) or out; device FP32 vectors. */
riot_status riot_sketchnet_set_params(riot_sketchnet *net, const float *params_dev);
riot_status riot_sketchnet_get_params(riot_sketchnet *net, float *params_dev);
/* Z (batch x m_out x n, i.e. m_out directions of n) from x (batch x c_in x n).  bf16 = 1
 * rounds weights and activations to BF16 (accumulation stays FP32). */
riot_status riot_sketchnet_forward(riot_sketchnet *net, const float *x_dev, int32_t n, int32_t batch, float *Z_dev,
                                   int32_t bf16);
/* Mean loss (host, may be NULL; synchronises) and its gradient (device, num_params
 * floats; NULL keeps it inside the network) for targets U (batch x r x n). */
riot_status riot_sketchnet_loss_grad(riot_sketchnet *net, const float *x_dev, const float *U_dev, int32_t r, int32_t n,
                                     int32_t batch, double mu, float *grad_dev, double *loss_out);
/* One Adam step on one batch; loss_out (may be NULL) receives the loss before the step. */
riot_status riot_sketchnet_train_step(riot_sketchnet *net, const float *x_dev, const float *U_dev, int32_t r, int32_t n,
                                      int32_t batch, double mu, float lr, double *loss_out);
/* Network input from a trajectory ((T+1) x n doubles, device): x (c_in x n floats) =
 * the snapshots at steps floor(c T / c_in), standardised by their common mean and
 * standard deviation.  Synchronises. */
riot_status riot_sketchnet_input(const double *traj_dev, int32_t T, int64_t n, int32_t c_in, float *x_dev,
                                 void *cuda_stream);
void riot_sketchnet_destroy(riot_sketchnet *net);

/* The stored FP64 trajectory ((T+1) x n doubles) of the last riot_outer_begin
 * (Lorenz-96 contexts). */
riot_status riot_get_trajectory(riot_ctx *ctx, double *traj_dev);

/* riot_rsvd with a proposed block: the m directions P_dev (m x n floats) are
 * orthonormalised into Q_p and the sketch is [Q_p, k - m Gaussian columns].
 * The proposal is kept only if its Rayleigh residual
 *   rho = ||A Q_p - Q_p (Q_p^T A Q_p)||_F / ||A Q_p||_F <= rho_max
 * (those products are part of the sketch); otherwise the sketch falls back to
 * k Gaussian columns, exactly as riot_rsvd.  rho_out (-1 when m = 0) and
 * used_out (1 if the proposal was kept) may be NULL.  Mixed precision only. */
riot_status riot_rsvd_proposal(riot_ctx *ctx, int32_t k, int32_t q, int64_t sketch_stream, const float *P_dev, int32_t m,
                               double rho_max, double *lambda_out, double *rho_out, int32_t *used_out);

/* Algorithm 1 (VarCG: conjugate gradients in Lanczos form, Section 2.1) with
 * full re-orthogonalisation, the sequential comparator of RIOT: m Lanczos
 * steps on A from q_1 = g / ||g|| (g from riot_outer_begin), one Hessian-vector
 * product each (the context's precision), T_m = tridiag(beta, alpha, beta) and
 * its eigenpairs (theta, Z) on the GPU, U = Q Z, and
 * dv = -U diag(1 / (1 + theta)) U^T g into dv_dev (n doubles; may be NULL; the
 * state x, v is not changed).  theta_out (host, m doubles; may be NULL) gets
 * the Ritz values in decreasing order, m_used (may be NULL) the number of steps
 * taken (fewer than m when the Krylov space is exhausted).  1 <= m <= kmax.
 * It reuses the inner-loop workspace: call riot_rsvd again before
 * riot_increment or riot_analysis_cov_lowrank.  Synchronises (one host read
 * per step, for the stopping test). */
riot_status riot_varcg(riot_ctx *ctx, int32_t m, double *dv_dev, double *theta_out, int32_t *m_used);

/* Algorithm 2 (VarBL): block Lanczos on A from l gradient samples, m block
 * steps (Section 2.1, block-Lanczos paragraph; Algorithm 2).  B0_dev holds the
 * samples b_j = L^T H_j^T R^-1 d_j + v + eps_b_j as n x l FP64 columns
 * (column-major, ld n, on the device; the caller forms them, e.g. with one
 * context per sample: riot_outer_begin at x + L eps_b_j on observations
 * y - sigma eps_obs_j, then riot_get_state's g plus eps_b_j).  Q_1 = orth(B0);
 * step i applies A to the l columns of Q_i (one batched launch), M_i = Q_i^T A Q_i,
 * r = A Q_i - Q_i M_i - Q_{i-1} W_{i-1}^T re-orthogonalised against Q_1..Q_i twice,
 * Q_{i+1} W_i = r by CholeskyQR (W_i = Q_{i+1}^T r).  The recurrence stops early
 * when a residual block loses rank (a diagonal entry of W_i at or below 1e-12
 * of the largest |M| entry so far, or a failed Cholesky): the block Krylov space
 * is then invariant.  T (block tridiagonal, M_i / W_i / W_i^T) = Z Theta Z^T,
 * U = Q Z, dv = -U diag(1 / (1 + theta)) U^T g with g the gradient of the
 * context (riot_outer_begin).  dv_dev (n, may be NULL): the increment;
 * theta_out (host, l m doubles, may be NULL): the Ritz values, descending, of
 * which the first l * blocks_used are written; blocks_used (may be NULL).
 * Requires riot_outer_begin (RIOT_ESTATE), 1 <= l m <= min(kmax, n)
 * (RIOT_EINVAL), no preconditioner factors (RIOT_ESTATE); RIOT_ENOTSPD if the
 * samples are linearly dependent.  Reuses the inner-loop workspace like
 * riot_varcg.  Synchronises (once per block step). */
riot_status riot_varbl(riot_ctx *ctx, int32_t l, int32_t m, const double *B0_dev, double *dv_dev, double *theta_out,
                       int32_t *blocks_used);

/* RIOT-PSAS (Appendix, Algorithm 4): one cycle of the observation-space dual
 * at the state of the last riot_outer_begin (either model).  With
 * S = L_{R^-1} = diag(1/sigma_o) (R diagonal) it decomposes the p x p
 * A_dual = S H B H^T S by the randomized steps of Algorithm 3 on a p x m
 * sketch (Omega_dev: p x m FP64 column-major on the device, or NULL to draw it
 * from sketch_stream; q power iterations; K from K Q^T W = Q^T Y, or
 * K = Q^T A_dual Q when the context was set up with exact_rr), then forms
 * the adaptive weights (lambda_m > 1: LRA, else LRU)
 *     dw = S U diag(1/(1+lambda)) U^T S (d - b')      or
 *     dw = S (I - U diag(lambda/(1+lambda)) U^T) S (d - b'),
 * d = y - H(x), b' = H (x_b - x) (tangent linear), and sets
 * x = x_b + B H^T dw, i.e. v = L^T H^T dw in the context's x = x_b + L v
 * (the listing writes x_{k-1} + B H^T dw, which counts x_{k-1} - x_b twice
 * from the second cycle on; both agree in the first).  Each product by
 * A_dual is one adjoint integration from the forcing S w, L L^T, and one
 * tangent-linear integration, in FP64 on either precision: Lorenz-96 one
 * launch of each over all m columns; the tracer model batches of the
 * columns its product workspace holds in FP64.
 * lambda_out (host, m, may be NULL): eigenvalues of A_dual, descending;
 * dv_dev (n, may be NULL): the change of v; mode_out (may be NULL): 0 LRA,
 * 1 LRU.  RIOT_ESTATE before riot_outer_begin or with preconditioner
 * factors; RIOT_EINVAL for m outside [1, min(kmax, p)] or q
 * outside [0, 64]; RIOT_ENOTSPD if the basis or the solve for K fails.
 * Allocates its observation-space workspace (6 p kmax doubles) at the first
 * call.  Synchronises.  Call riot_outer_begin() before the next cycle. */
riot_status riot_psas(riot_ctx *ctx, int32_t m, int32_t q, int64_t sketch_stream, const double *Omega_dev,
                      double *lambda_out, double *dv_dev, int32_t *mode_out);

/* Spectral preconditioner with rotation (Section 2.2 "Preconditioning", Eq. 7;
 * Algorithm 3 with precond = true).  After outer loop j has run riot_rsvd and
 * riot_increment, riot_precond_push(ctx, m) adds the factor
 *     P'_j = I + V_j ((Lambda_j + I)^-1/2 - I) V_j^T
 * built from that loop's leading m Ritz pairs (V_j = the first m columns of U,
 * Lambda_j their eigenvalues of the preconditioned Hessian).  Every later loop k
 * then runs with P_k = P'_1 ... P'_{k-1}:
 *   - riot_outer_begin sets g = P_k^T (b + v)       (v stays the control of
 *     x = x_b + L v: the problem of loop k is solved for w with v = v_{k-1} + P_k w);
 *   - riot_rsvd decomposes A_k = P_k^T P_k - I + P_k^T A P_k instead of A (its
 *     eigenvalues and Ritz vectors are those of A_k);
 *   - riot_increment forms the adaptive increment dw of Algorithm 3 from g and
 *     the pairs of A_k, then v += P_k dw and x += L P_k dw (dv_dev receives P_k dw).
 * With rotation on, riot_rsvd first projects every sketch column (drawn or
 * given) onto the orthogonal complement of the span of [P_1 V_1, ..., P_{k-1}
 * V_{k-1}] (Algorithm 3's (I - U_k U_k^T); its following P_k^-1 is the identity
 * on that complement and is not applied), and requires k + (resolved columns) <= n.
 * After a push, riot_outer_begin must run before the next riot_rsvd or
 * riot_increment (RIOT_ESTATE otherwise): the gradient depends on P_k.
 * riot_varcg, riot_rsvd_proposal and batches refuse contexts with factors
 * (RIOT_ESTATE / RIOT_EINVAL).
 *
 * The solve for K of Algorithm 3 can return trailing Ritz values below -1 on
 * the flattened spectrum of a preconditioned loop; (Lambda + I)^-1/2 is then
 * undefined, so push the leading pairs with positive eigenvalue (the
 * benchmark and the tests take m = the number of positive values).
 *
 * riot_precond_enable(ctx, max_cols, rotation): drops all factors and reserves
 * device storage for max_cols stored columns in total (0 <= max_cols <= n;
 * 0 switches the preconditioner off and frees it); synchronises the stream.
 * riot_precond_push: RIOT_ESTATE before riot_precond_enable, or unless
 * riot_increment ran after the last riot_rsvd (one push per outer loop);
 * RIOT_EINVAL if m is outside [1, k] or the storage is full; RIOT_ENONFINITE if
 * an eigenvalue of I + A_k is not positive; RIOT_ENOTSPD if the new rotation
 * directions are dependent on the old ones.  Synchronises.
 * riot_precond_push_pairs(ctx, V, lambda, m): the same factor from given pairs
 * (a preconditioner kept from an earlier cycle, or pairs computed elsewhere):
 * V n x m FP64 on the device (column-major, ld n, orthonormal columns),
 * lambda m host values (eigenvalues of the Hessian the factor preconditions);
 * 1 <= m <= kmax.  RIOT_ESTATE between a riot_rsvd and its riot_increment;
 * otherwise as riot_precond_push.
 * riot_precond_apply(ctx, X, Y, ncols, op): Y = op(P_k) X for ncols FP64
 * columns of length n (column-major, ld n; X == Y allowed), op 0 = P_k,
 * 1 = P_k^T, 2 = P_k^-1.  Asynchronous on the context stream.
 * riot_precond_count: the number of factors (-1 for a null context). */
riot_status riot_precond_enable(riot_ctx *ctx, int32_t max_cols, int32_t rotation);
riot_status riot_precond_push(riot_ctx *ctx, int32_t m);
riot_status riot_precond_push_pairs(riot_ctx *ctx, const double *V_dev, const double *lambda, int32_t m);
riot_status riot_precond_apply(riot_ctx *ctx, const double *X_dev, double *Y_dev, int32_t ncols, int32_t op);
int32_t riot_precond_count(const riot_ctx *ctx);

/* The FP32 sketch GEMM of the mixed-precision path on its own, for checks:
 * C = alpha op(A) op(B) + beta C (column-major FP32, op 'N' or 'T') on the
 * tcgen05 tensor cores, each operand split into three BF16 terms and the six
 * leading term products accumulated in FP32 (FP32 accuracy).  Allocates and
 * frees its own workspace; synchronises the stream.  RIOT_ETIMEOUT if a
 * bounded wait on the tensor cores ran out. */
riot_status riot_tc_sgemm(char ta, char tb, int32_t m, int32_t n, int32_t k, float alpha, const float *A_dev,
                          int64_t lda, const float *B_dev, int64_t ldb, float beta, float *C_dev, int64_t ldc,
                          void *cuda_stream);

/* The Gram matrix of the mixed-precision CholeskyQR (Section 2.2, the
 * orthonormalisation Q = orth(Y) of Algorithm 3) on its own, for checks: the
 * lower triangle (i >= j) of G = Y^T Y, Y n x k FP32 column-major (leading
 * dimension ldy >= n), G k x k FP64 column-major (ldg >= k; the strict upper
 * triangle is not written).  Computed on the tcgen05 tensor cores by exact
 * integer slicing: each column is scaled by a power of two and split into five
 * BF16 slices whose products and sums are exact, so the only error off the
 * diagonal is the truncation of each value below 2^-36 of its column's largest
 * magnitude (and the slice products of weight below 2^-42 that are left out);
 * the diagonal is summed in FP64 on the CUDA cores.  A column
 * holding Inf or NaN gives NaN in its row and column of G.  n = 0 gives G = 0.
 * Allocates and frees its own workspace; synchronises the stream.
 * RIOT_ETIMEOUT if a bounded wait on the tensor cores ran out. */
riot_status riot_tc_gram(int32_t n, int32_t k, const float *Y_dev, int64_t ldy, double *G_dev, int64_t ldg,
                         void *cuda_stream);

const char *riot_last_error(const riot_ctx *ctx);
const char *riot_status_string(riot_status s);
void riot_destroy(riot_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* RIOT_H */
