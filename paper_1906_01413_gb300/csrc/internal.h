// Internal declarations shared by the translation units of the RIOT library.
// Nothing here is part of the public C ABI (include/riot.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/riot.h"

namespace riot {

// ---------------------------------------------------------------------------
// Chunked layout of one Lorenz-96 state across the threads that own it.
// Thread t of a probe holds len(t) consecutive variables starting at
// start(t); len is E for the first Tp-g threads and E-1 for the last g.
// Per-thread arrays ("slots") are padded to E: slot = t*E + j.
// ---------------------------------------------------------------------------
struct ChunkGeom {
    int n = 0;   // variables
    int E = 0;   // elements per thread (template parameter of the kernels)
    int Tp = 0;  // threads per probe
    int g = 0;   // number of short (E-1) chunks, at the end
    int Np = 0;  // Tp*E
    __host__ __device__ int start(int t) const {
        int over = t - (Tp - g);
        return t * E - (over > 0 ? over : 0);
    }
    __host__ __device__ int len(int t) const { return t < Tp - g ? E : E - 1; }
    // slot of variable i
    __host__ __device__ int slot(int i) const {
        int full = (Tp - g) * E;
        if (i < full) return i;
        int r = i - full;
        int t = (Tp - g) + r / (E - 1);
        return t * E + r % (E - 1);
    }
};

// Pick E in {4, 8, 16} and fill the geometry; returns false if n is out of range.
bool choose_geom(int n, ChunkGeom *geom);

// Gaussian square-root band (L = diag(sigma) S, S symmetric circulant):
// S_d for d in [-hl, hh], stored at band[d + hl].
struct Band {
    int hl = 0, hh = 0;
};

// ---------------------------------------------------------------------------
// Lorenz-96 kernels (l96.cu)
// ---------------------------------------------------------------------------
struct L96Dev {
    ChunkGeom geom;
    int T = 0;
    double dt = 0, F = 0;
    // observations, sorted by step
    int p = 0;
    const int *optr = nullptr;    // [T+2]: obs of step t are optr[t] .. optr[t+1]-1
    const int *oslot = nullptr;   // [p] slot of the observed variable
    const int *oidx = nullptr;    // [p] observed variable
    const double *y = nullptr;    // [p]
    const double *rinv64 = nullptr;  // [p] 1/sigma^2
    const float *rinv32 = nullptr;
    // prior square root
    Band band;
    const double *band64 = nullptr;
    const float *band32 = nullptr;
    const double *sig64 = nullptr;   // [n]
    const float *sig32 = nullptr;
    // warp-synchronous FP32 Hessian kernel (l96_warp.cu): observations sorted by
    // (step, slot) with each thread's range per observed step, and the stage
    // coefficients in per-warp blocks
    const int *ostep = nullptr;      // [T+1] index of step t among the observed steps, -1 if none
    const int *ostart = nullptr;     // [observed steps][Tp+1] first sorted observation of each chunk
    const int *osslot = nullptr;     // [p] slot of each sorted observation
    const int *osperm = nullptr;     // [p] index of each sorted observation in the caller's order
};

// Nonlinear FP64 trajectory of one state; writes traj (T+1)*n (natural
// layout, may be null), stage coefficients (may be null): double2 by slot
// t*E + j, and float2 interleaved by element pair ((j/2)*Tp + t as float4),
// the innovation d = H(x) - y (may be null) and 1/2 sum d^2/sigma^2 into
// *jo (may be null, accumulated with atomicAdd: zero it first).
cudaError_t l96_nl_launch(const L96Dev &m, const double *x0, double *traj, float2 *coef32,
                          double2 *coef64, double *d, double *jo, double *xT, cudaStream_t s);

// Batched FP64 Hessian-vector product (register-loaded coefficients, layout
// [T][4][Np] double2 by slot).  mode 0: Y = A W (+W); mode 1: adjoint only
// with the given forcing r (one column, length p): Y = L^T lambda_0;
// mode 2: tangent linear only: r = R^-1 H M L W.
cudaError_t l96_hvp_launch_f64(const L96Dev &m, const double2 *coef, const double *W, double *Y,
                               int64_t ld, int ncols, int add_identity, double *r, int mode,
                               cudaStream_t s);

// FP32 Hessian-vector product with the stage coefficients streamed into
// shared memory by 1-D TMA copies (same modes as above); *err is raised to 1
// if a bounded wait on a copy ran out, to 2 if a copy was still in flight when
// its CTA exited after that.  wait_polls < 0: the default bound of each wait
// (about 2^20 polls); >= 0: that many polls (tests of the timeout report).
cudaError_t l96_hvp_tma_launch(const L96Dev &m, const float2 *coef, const float *W, float *Y, int64_t ld,
                               int ncols, int add_identity, float *r, int mode, int *err, cudaStream_t s,
                               int P_hint = 0, int S_hint = 0, int wait_polls = -1, bool two_per_sm = false);

// Warp-synchronous FP32 Hessian product (Y = A W (+W)): halos by warp shuffles and
// per-warp mailboxes, coefficients by per-warp 1-D TMA rings.  Needs E of 8 or 16 and
// 64 <= Tp <= 512 (warp_kernel_fits).  coefw holds l96_coef_warp_floats4 float4 written
// by l96_coef_warp from the FP64 stage coefficients; r holds ncols x p residuals (in the
// sorted observation order).  S_hint: ring depth (0: deepest that fits).
bool warp_kernel_fits(const ChunkGeom &g);
int warp_probes_per_cta(int E);
cudaError_t l96_warp_tables(const ChunkGeom &g, int T, const std::vector<int> &optr, const std::vector<int> &oslot,
                            std::vector<int> &ostep, std::vector<int> &ostart, std::vector<int> &sslot,
                            std::vector<int> &perm);
size_t l96_coef_warp_floats4(const L96Dev &m);
cudaError_t l96_coef_warp(const L96Dev &m, const double2 *coef64, float4 *coefw, cudaStream_t s);
cudaError_t l96_hvp_warp_launch(const L96Dev &m, const float4 *coefw, const float *W, float *Y, int64_t ld, int ncols,
                                int add_identity, float *r, int *err, cudaStream_t s, int S_hint = 0,
                                int wait_polls = -1, bool shuffle = false);

// Several Lorenz-96 windows' FP32 Hessian products (Y = A W) in one
// persistent launch over a queue of (window, CTA block) items.
struct HvpBatchWindow {
    const L96Dev *m;
    const float2 *coef;
    const float *W;
    float *Y;
    int64_t ld;
    int ncols;
    float *r;
    int *err;
};
struct HvpBatchPlan {
    int nwin = 0, nitems = 0, grid = 0, nthr = 0, P_cap = 0, S = 0;
    size_t smem = 0;
    void *d_args = nullptr, *d_items = nullptr;
    int *d_counter = nullptr;
};
// P_cap caps the probe groups per CTA (0: as many as fit), S the ring depth
// (0: 4, lowered per window to fit shared memory).  Allocates device tables.
cudaError_t hvp_batch_plan(const HvpBatchWindow *w, int nwin, int P_cap, int S, HvpBatchPlan *plan);
cudaError_t hvp_batch_launch(const HvpBatchPlan &plan, cudaStream_t s);
void hvp_batch_free(HvpBatchPlan *plan);

// out = L in or L^T in (FP64), ncols columns (ld = n)
cudaError_t bsqrt_launch(const L96Dev &m, const double *in, double *out, int transpose, int ncols,
                         cudaStream_t s);

// ---------------------------------------------------------------------------
// Tracer transport model (advdiff.cu)
// ---------------------------------------------------------------------------
struct AdvDev {
    int nx = 0, ny = 0, nz = 0, nb = 0, T = 0;
    double dt = 0, dx = 0, dy = 0, dz = 0, sigma_b = 0;
    long long n = 0, ncells = 0;
    int p = 0;
    std::vector<int> optr_h;          // host copy [T+2]: obs of step t are optr[t] .. optr[t+1]-1
    std::vector<double> amp_h, kz_h;  // host copies [nz], [nz+1] (kernel parameters)
    const int *cell = nullptr;        // [p*8] flat cell (l*ny + j)*nx + i of each trilinear corner
    const double *w64 = nullptr;      // [p*8] trilinear weights
    const float *w32 = nullptr;
    const double *y = nullptr, *rinv64 = nullptr;
    const float *rinv32 = nullptr;
    const double *u64 = nullptr, *v64 = nullptr, *amp64 = nullptr, *kz64 = nullptr;
    const float *u32 = nullptr, *v32 = nullptr, *amp32 = nullptr, *kz32 = nullptr;
    const double *Sx64 = nullptr, *Sy64 = nullptr;   // symmetric square roots, row-major
    const float *Sx32 = nullptr, *Sy32 = nullptr;
    const double *Eb = nullptr;       // [n] background emissions
    double *Es64 = nullptr;           // [n] E / dz at the current control
    float *Es32 = nullptr;
    // batch workspace (Pmax probes of the context precision; the same bytes hold Pws64 FP64 probes)
    int Pmax = 0, Pmax64 = 0, Pws64 = 0;
    void *cA = nullptr, *cB = nullptr, *src = nullptr, *ebar = nullptr, *tmp = nullptr;
    // FP64 outer-loop workspace
    double *c64A = nullptr, *c64B = nullptr, *ebar64 = nullptr, *tmp64 = nullptr;   // tmp64: Pmax64 * n
};

// Y = A W (+ W) for ncols columns (ld >= n), in FP64 or FP32 (per fp64); r
// holds Pmax * p residuals of that type.
cudaError_t adv_hvp(const AdvDev &m, bool fp64, const void *W, void *Y, int64_t ld, int ncols, int add_identity,
                    void *r, cudaStream_t s);
// Outer-loop prerequisites at control x (FP64): E / dz, d = H(x) - y,
// jo += 1/2 sum d^2 / sigma^2 (atomic), rd = R^-1 d, b = L^T H'^T R^-1 d.
cudaError_t adv_outer(const AdvDev &m, const double *x, double *d, double *jo, double *rd, double *b,
                      cudaStream_t s);
// The halves of a product in FP64 on either precision, over ncols columns (Pws64 at a time, in
// the batch workspace): the tangent linear r = R^-1 H' L w (W at ld, r: ncols x p) and the
// adjoint z = L^T H'^T f from an observation-space forcing (f: ncols x p, Z at ld); for the
// dual of Algorithm 4.
cudaError_t adv_tl(const AdvDev &m, const double *W, int64_t ld, int ncols, double *r, cudaStream_t s);
cudaError_t adv_ad(const AdvDev &m, const double *f, int ncols, double *Z, int64_t ld, cudaStream_t s);
// z = L^T H'^T f for one FP64 observation-space forcing (outer-loop workspace)
cudaError_t adv_ad_obs(const AdvDev &m, const double *f, double *z, cudaStream_t s);
// Tangent-linear observation residuals of one FP64 column w: r = R^-1 H' (L w), the forward
// half of a Hessian product (uses the outer-loop workspace; p doubles out).
cudaError_t adv_tl_obs(const AdvDev &m, const double *w, double *r, cudaStream_t s);
// out = L in (= L^T in), ncols columns of n doubles
cudaError_t adv_bsqrt(const AdvDev &m, const double *in, double *out, int ncols, cudaStream_t s);
// tracer field after `steps` steps from zero with emissions E_b exp(x) (FP64)
cudaError_t adv_forecast(const AdvDev &m, const double *x, int steps, double *c_out, cudaStream_t s);

// ---------------------------------------------------------------------------
// Learned sketch proposal (sketchnet.cu)
// ---------------------------------------------------------------------------
struct SketchNet {
    int c_in = 0, width = 0, m = 0, depth = 0, K = 0;
    int chan[9] = {0};   // channels of layer inputs/outputs: c_in, width .. width, m
    int64_t num_params() const;
    int64_t w_offset(int l) const;   // offset of layer l's weights in the flat vector
};
struct SketchWork {
    float *Z = nullptr, *acts = nullptr, *gZ = nullptr, *g0 = nullptr, *g1 = nullptr;
    float *R = nullptr, *UtX = nullptr, *G = nullptr, *E = nullptr, *XE = nullptr;
    double *sc = nullptr;   // 4 doubles per window
};
// Z (B x m x n) from x (B x c_in x n); hidden activations into acts ((depth-1) x B x width x n)
cudaError_t sketchnet_forward(const SketchNet &net, const float *params, const float *x, int n, int B, float *Z,
                              bool bf16, float *acts, cudaStream_t s);
// mean subspace loss over B windows (targets U: B x r x n, orthonormal columns) into *loss_dev
// and its parameter gradient into grad
cudaError_t sketchnet_loss_grad(const SketchNet &net, const float *params, const float *x, const float *U, int r,
                                int n, int B, double mu, float *grad, double *loss_dev, SketchWork &w,
                                cudaStream_t s);
cudaError_t sketchnet_adam(const SketchNet &net, float *params, const float *grad, float *m1, float *m2, int t,
                           float lr, cudaStream_t s);
// x (C x n) = standardised snapshots of traj ((T+1) x n, FP64) at steps floor(c T / C); st: 2 doubles
cudaError_t sketchnet_input(const double *traj, int T, int64_t n, int C, float *x, double *st, cudaStream_t s);
// out[0] += sum of squares of x (double accumulation)
cudaError_t sumsq(const float *x, size_t n, double *out, cudaStream_t s);

// ---------------------------------------------------------------------------
// Random numbers (rng.cu)
// ---------------------------------------------------------------------------
cudaError_t normal_launch(uint64_t seed, uint32_t stream, int64_t n, int ncols, int64_t ld,
                          int is_double, void *out, cudaStream_t s);

// ---------------------------------------------------------------------------
// Dense linear algebra, column-major (linalg.cu)
// ---------------------------------------------------------------------------
// C = alpha op(A) op(B) + beta C with double accumulation.
// Types: 'f' float, 'd' double for A, B and C.
cudaError_t gemm(char ta, char tb, int m, int n, int k, double alpha, const void *A, char tA,
                 int64_t lda, const void *B, char tB, int64_t ldb, double beta, void *C, char tC,
                 int64_t ldc, cudaStream_t s);
// lower-triangular tiles of G = A^T A (A: n x k), the rest of G untouched
cudaError_t gram_lower(int n, int k, const void *A, char tA, int64_t lda, double *G, int64_t ldg, cudaStream_t s,
                       double *ws = nullptr, size_t ws_doubles = 0);
// FP32 SIMT GEMM, C = alpha op(A) op(B) + beta C
cudaError_t sgemm(char ta, char tb, int m, int n, int k, float alpha, const float *A, int64_t lda, const float *B,
                  int64_t ldb, float beta, float *C, int64_t ldc, cudaStream_t s);
// FP32-accurate GEMM on tcgen05 tensor cores (three BF16 terms per value, six MMAs per
// K step, FP32 accumulation in tensor memory): C = alpha op(A) op(B) + beta C,
// column-major.  ws (tc_sgemm_ws_floats floats, may be null) holds split-K partial tiles;
// err is set if a bounded wait on the MMAs ran out.
cudaError_t tc_sgemm(char ta, char tb, int m, int n, int k, float alpha, const float *A, int64_t lda, const float *B,
                     int64_t ldb, float beta, float *C, int64_t ldc, float *ws, size_t ws_floats, int *err,
                     cudaStream_t s);
size_t tc_sgemm_ws_floats(int m, int n, int k);
// Lower triangle of G = Y^T Y (Y: n x k FP32, column-major) to FP64-level
// accuracy on the tensor cores (error-free slicing, exact integer
// accumulation, FP64 diagonal).  ws: tc_gram_ws_bytes(k) bytes of device
// memory, 16-byte aligned; err is set if a bounded wait on the tensor cores ran out.
cudaError_t tc_gram_f32(int n, int k, const float *Y, int64_t ldy, double *G, int64_t ldg, void *ws, int *err,
                        cudaStream_t s);
size_t tc_gram_ws_bytes(int k);
// X <- X L^-T in FP32 (L: k x k lower, FP32)
// Diagonal 32 x 32 blocks of L32 replaced by the FP32 rounding of the block
// inverses dinv that cholesky leaves; strsm_right_lt_inv then solves
// X <- X L^-T with products by those inverses (no substitution chains).
cudaError_t put_block_inverses(float *L32, int k, int64_t ldl, const double *dinv, cudaStream_t s);
cudaError_t strsm_right_lt_inv(float *X, int m, int k, int64_t ldx, const float *L, int64_t ldl, cudaStream_t s);
cudaError_t convert_block(const void *in, char tin, int64_t ldin, void *out, char tout, int64_t ldout,
                          int64_t rows, int cols, cudaStream_t s);
// In-place blocked Cholesky of the k x k SPD matrix G (lower factor); adds
// shift_scale * trace(G) to the diagonal first when shift_scale > 0.
// info[0] = 0 on success, else 1 + first failing pivot (-1: a bounded wait of the
// cooperative form ran out).  dinv (dinv_doubles(k))
// receives the inverses of the factor's 32 x 32 diagonal blocks, which the
// triangular solves below use.  whole_gpu: one cooperative launch over every SM
// (the GPU runs nothing else meanwhile: a single window); else two launches per
// block column with small grids, which windows on parallel streams can share.
cudaError_t cholesky(double *G, int k, int64_t ldg, double shift_scale, int *info, double *dinv, cudaStream_t s,
                     bool whole_gpu = true);
size_t dinv_doubles(int k);
// inverses of the diagonal blocks of a lower-triangular L (when not from cholesky)
cudaError_t trtri_diag(const double *L, int k, int64_t ldl, double *dinv, cudaStream_t s);
// C (lower triangle) = A A^T, A n x K, FP64
cudaError_t syrk_lower(int n, int K, const double *A, int64_t lda, double *C, int64_t ldc, cudaStream_t s);
// X <- X L^-T (X: m x k, L: k x k lower): right-side solve with diagonal-block inverses.
cudaError_t trsm_right_lt(double *X, int m, int k, int64_t ldx, const double *L, int64_t ldl, cudaStream_t s,
                          const double *dinv);
// X <- X L^-1 (L lower, non-unit): right-side solve with diagonal-block inverses.
cudaError_t trsm_right_l(double *X, int m, int k, int64_t ldx, const double *L, int64_t ldl, cudaStream_t s,
                         const double *dinv);
// Symmetric eigendecomposition by parallel cyclic Jacobi (cooperative
// launch).  A (k x k, ld = k) is destroyed; lam gets eigenvalues sorted in
// decreasing order, Z (k x k, ld = k) the eigenvectors with the
// largest-magnitude entry of each made positive.  work: 3*k*k + 64 doubles
// (ke = k rounded up to even).  info[0] = number of sweeps (< 0: no convergence).
cudaError_t jacobi_eig(double *A, int k, double *lam, double *Z, double *work, int *info,
                       cudaStream_t s);
size_t jacobi_work_doubles(int k);
// Symmetric eigendecomposition by Householder tridiagonalisation, bisection
// and inverse iteration (all SMs; O(k) grid barriers).  K is not modified.
// lam: eigenvalues descending; Z (k x k): eigenvectors.  info[0..1] != 0 if
// the final orthonormalisation of the eigenvectors failed.
// fp32_vectors: the eigenvectors are consumed in FP32, so their orthonormalisation
// stops at about 1e-7 (one shifted CholeskyQR pass less); with tc_err (the flag of the
// tensor-core kernels' bounded waits) it runs on their FP32 rounding with the exact
// tensor-core Gram and the one-launch FP32 solve, as the mixed path's CholeskyQR does
cudaError_t tridiag_eig(const double *K, int k, double *lam, double *Z, double *work, int *info, cudaStream_t s,
                        bool fp32_vectors = false, int *tc_err = nullptr);
size_t eig_work_doubles(int k);
// elementwise helpers
cudaError_t symmetrize(double *A, int k, int64_t lda, cudaStream_t s);
cudaError_t transpose_sq(const double *A, double *B, int k, cudaStream_t s);
cudaError_t axpby(int64_t n, double a, const double *x, double b, double *y, cudaStream_t s);
// increment helper: c (k) -> scaled coefficients by mode over the retained pairs (the
// leading m with lam_i >= rel_floor lam_0; all k when rel_floor < 0); writes the mode to
// mode_dev[0] and m to mode_dev[1]
cudaError_t increment_coef(const double *lam, int k, double *c, int *mode_dev, double rel_floor, cudaStream_t s);
cudaError_t cov_coef(const double *lam, int m, double *coef, int *mode_dev, cudaStream_t s);
cudaError_t check_finite(const double *x, int64_t n, int *flag, cudaStream_t s);
// y += a x when flag[0] == want (flag read on the device)
cudaError_t add_if_flag(const int *flag, int want, int64_t n, double a, const double *x, double *y, cudaStream_t s);
cudaError_t mul(int64_t n, const double *a, const double *b, double *out, cudaStream_t s);
cudaError_t add_half_sq(int64_t n, const double *x, double *out, cudaStream_t s);
// out += 1/2 sum (d + r / rinv)^2 rinv over p observations (r may be null: 1/2 sum d^2 rinv)
cudaError_t obs_quad_cost(int64_t p, const double *d, const double *r, const double *rinv, double *out, cudaStream_t s);
cudaError_t scale_to_f32(int64_t n, const double *in, double a, float *out, cudaStream_t s);
// Column equilibration of one CholeskyQR pass: with d_j = 1/sqrt(G_jj),
// G <- D G D (lower triangle) and Q <- Q D ('f' or 'd' block, n rows); d receives D.
cudaError_t equilibrate(double *G, int k, int64_t ldg, void *Q, char tQ, int64_t n, int64_t ldq, double *d,
                        cudaStream_t s);
cudaError_t scal(int64_t n, double a, double *x, cudaStream_t s);
// vector steps of the Lanczos form of conjugate gradients (Algorithm 1)
cudaError_t dot_dev(int64_t n, const double *x, const double *y, double *out, cudaStream_t s);
cudaError_t lanczos_resid(int64_t n, const double *w, const double *q, const double *qprev, const double *alpha,
                          double beta_prev, double *r, cudaStream_t s);
cudaError_t normalize_by(int64_t n, const double *r, const double *rr, double *q, cudaStream_t s);
cudaError_t tridiag_fill(int m, const double *alpha, const double *beta, double *T, cudaStream_t s);
cudaError_t div_one_plus(int m, double *c, const double *theta, cudaStream_t s);
// block Lanczos (Algorithm 2): T (nb l square, ld nb l) from the blocks M_i (at blocks + i l^2)
// and W_i (at blocks + (mcap + i) l^2), each l x l column-major
cudaError_t block_tridiag_fill(int nb, int l, int mcap, const double *blocks, double *T, cudaStream_t s);
// Y = a Y (+ W) column by column (n rows of ncols columns at ld), float or double
cudaError_t scale_add_cols(int64_t n, int ncols, int64_t ld, double a, void *Y, const void *W, int is_double,
                           cudaStream_t s);
// T (m x ncols at ld, float or double) with row i scaled by coef[i]
cudaError_t scale_rows(int m, int ncols, int64_t ld, const double *coef, void *T, int is_double, cudaStream_t s);
// Y = a X + b Y on n rows of ncols columns at ld, float or double
cudaError_t axpby_cols(int64_t n, int ncols, int64_t ld, double a, const void *X, double b, void *Y, int is_double,
                       cudaStream_t s);
// out[:, j] = in[:, perm[j]] for m columns of n doubles (perm on the device; out must not alias in)
cudaError_t gather_cols(const double *in, int64_t ldi, const int *perm, int m, int64_t n, double *out, int64_t ldo,
                        cudaStream_t s);
// largest-magnitude entry of each of the k columns made positive
cudaError_t fix_col_signs(double *U, int64_t n, int k, int64_t ld, cudaStream_t s);

int num_sms();
// host-side count of kernel launches issued by the library
void count_launch();
unsigned long long launches_total();

}  // namespace riot
