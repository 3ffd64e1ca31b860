// C ABI of the RIOT inner-loop library (see include/riot.h for the contract).
//
// Host orchestration only: every arithmetic step of the inner loop runs in
// the kernels of l96.cu, rng.cu and linalg.cu on the context's stream.  The
// host builds the model tables once in riot_setup (observation pointers and
// slots, the banded Gaussian square-root kernel) and then only launches.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "internal.h"

using namespace riot;

// One buffer a context owns, with its size (the caller's allocator may want it back).
struct riot_alloc_rec {
    void *p;
    size_t bytes;
};

struct riot_ctx {
    int dev = 0;
    int model = RIOT_MODEL_L96;
    int n = 0, p = 0;   // control size, observation count
    cudaStream_t s = nullptr;
    int prec = RIOT_PREC_MIXED;
    int kmax = 0, exact_rr = 0, eig_method = 0;
    int hvp_P = 0, hvp_S = 0;   // launch shape of the FP32 Hessian kernel (0 = automatic)
    uint64_t seed = 0;
    L96Dev m;
    AdvDev a;   // tracer model (RIOT_MODEL_ADVDIFF)
    // device allocator of riot_options (NULL: cudaMalloc / cudaFree) and what it gave out
    riot_dev_alloc_fn dev_alloc = nullptr;
    riot_dev_free_fn dev_free = nullptr;
    void *alloc_user = nullptr;
    std::vector<riot_alloc_rec> allocs;
    int wait_polls = -1;   // poll bound of the Hessian kernel's waits (-1: default; riot_set_wait_limit)
    // model tables
    int *optr = nullptr, *oslot = nullptr, *oidx = nullptr;
    double *y = nullptr, *rinv64 = nullptr, *band64 = nullptr, *sig64 = nullptr;
    float *rinv32 = nullptr, *band32 = nullptr, *sig32 = nullptr;
    // outer-loop state
    double *x = nullptr, *v = nullptr, *g = nullptr, *dv = nullptr, *tmp = nullptr;
    double *v0 = nullptr;   // v at the last riot_outer_begin (the quadratic cost's control)
    double *xsave = nullptr, *vsave = nullptr;   // x, v before a batched inner loop (to redo one window)
    double *traj = nullptr, *d = nullptr, *rd = nullptr, *jo = nullptr;
    float2 *coef32 = nullptr;
    double2 *coef64 = nullptr;
    float4 *coefw = nullptr;   // per-warp FP32 stage coefficients of the warp-synchronous kernel (mixed)
    int hvp_kernel = RIOT_HVP_CTA_BARRIER;   // FP32 Hessian kernel (riot_set_hvp_kernel)
    // inner-loop workspace
    void *Wblk = nullptr, *Yblk = nullptr, *rscr = nullptr;
    double *Q = nullptr, *U = nullptr;
    float *Q32 = nullptr, *M32 = nullptr, *N32 = nullptr, *L32 = nullptr;   // mixed precision only
    float *tcws = nullptr;   // split-K workspace of the tensor-core sketch GEMMs
    size_t tcws_floats = 0;
    double *G = nullptr, *Mm = nullptr, *Nm = nullptr, *Km = nullptr, *Z = nullptr, *lam = nullptr, *cvec = nullptr;
    double *jwork = nullptr;
    double *gws = nullptr;   // split-K partial Grams (8 kmax^2) and Cholesky block inverses (dinv_doubles(kmax))
    int *info = nullptr;  // [0..9] CholeskyQR passes, [10] K Cholesky, [12..13] Jacobi, [14] mode
    int *errflag = nullptr;  // set by a kernel whose bounded wait ran out
    int have_traj = 0, have_rsvd = 0, k_last = 0, v_init = 0, jacobi_sweeps = 0;
    // deflated two-level eigendecomposition (riot_rsvd_deflated), allocated at its first call:
    // the level-1 Ritz vectors kept (FP64 and FP32), then the combined pairs before sorting
    int deflated = 0;   // the current pairs came from riot_rsvd_deflated (all are retained)
    double *Ud64 = nullptr;
    float *Ud32 = nullptr;
    int *perm = nullptr;
    // FP32 Hessian products are formed as 2^-scale_exp A (R^-1 scaled by 2^-scale_rinv in
    // rinv32, the input and output by 2^-scale_in through sig32) so that windows whose
    // tangent-linear growth exceeds the FP32 range stay finite; eigenvalues are scaled
    // back in FP64.
    int scale_exp = 0, scale_in = 0, scale_rinv = 0;
    int k_shift = 0;   // shift the K normal equations (set for one retry after a failed solve)
    int qr_shift_all = 0;   // every FP64 CholeskyQR pass shifted (set for one retry of a rank-deficient block)
    double *nrm = nullptr;   // 4 doubles of norm accumulators
    // Spectral preconditioner of Algorithm 3 (riot_precond_*): P_k = P'_1 ... P'_{k-1},
    // P'_j = I + V_j diag(c_j) V_j^T with c_j = (lambda_j + 1)^-1/2 - 1 (its inverse takes
    // ci_j = (lambda_j + 1)^1/2 - 1); factor j holds pc_m[j] columns from column pc_off[j].
    int pc_cap = 0, pc_rot = 0, pc_cols = 0, rot_cols = 0;
    int pc_ready = 0;   // riot_increment ran since the last riot_rsvd (and no push since)
    int pc_open = 0;    // riot_rsvd finished, its riot_increment not yet run
    int pc_dirty = 0;   // a factor was added after riot_outer_begin formed g with the old P_k
    std::vector<int> pc_off, pc_m;
    double *pcV = nullptr, *pcc = nullptr, *pci = nullptr, *pcT = nullptr;
    double *pcB = nullptr;   // rotation: orthonormal basis of [P_1 V_1, ..., P_{k-1} V_{k-1}] (rot_cols columns)
    float *pcV32 = nullptr, *pcB32 = nullptr, *pcT32 = nullptr;   // FP32 copies (mixed precision)
    std::vector<riot_alloc_rec> pc_allocs;
    // RIOT-PSAS (riot_psas), allocated at its first call: observation-space blocks (p x kmax
    // FP64: sketch / basis input, products, basis, Ritz vectors, adjoint forcing, TL output),
    // S = diag(1 / sigma_o) and sigma_o, and p-vectors
    double *psW = nullptr, *psY = nullptr, *psQ = nullptr, *psU = nullptr, *psF = nullptr, *psR = nullptr;
    double *psS = nullptr, *psSig = nullptr, *psr = nullptr, *psw = nullptr, *psc = nullptr;
    // Cholesky factorisations as one cooperative launch over every SM (cleared while a batch
    // runs the windows' linear algebra on parallel streams)
    bool chol_whole_gpu = true;
    // timing
    cudaEvent_t ev[32];
    int nev = 0;
    int ev_phase[32];
    char err[512] = {0};
};

// A batch of Lorenz-96 windows run together (riot_batch_*).
struct riot_batch {
    int dev = 0;
    cudaStream_t s = nullptr;              // caller's stream
    cudaStream_t main = nullptr;           // the batch's own stream: main branch of the graph
    cudaEvent_t done = nullptr;
    std::vector<riot_ctx *> ctx;
    std::vector<int> k;
    int q = 0;
    std::vector<cudaStream_t> ws;          // one branch stream per window
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> join;
    std::vector<riot::HvpBatchWindow> wins;
    riot::HvpBatchPlan plan;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int64_t graph_sketch = -1;
    char err[512] = {0};
};

// A learned sketch network with its optimiser state and workspace (riot_sketchnet_*).
struct riot_sketchnet {
    int dev = 0;
    cudaStream_t s = nullptr;
    riot::SketchNet net;
    riot::SketchWork w;
    int n_max = 0, b_max = 0, r_max = 0, t = 0;
    float *params = nullptr, *grad = nullptr, *m1 = nullptr, *m2 = nullptr;
    double *loss = nullptr;
    std::vector<void *> allocs;
};

namespace {

riot_status fail(riot_ctx *c, riot_status st, const char *fmt, ...)
{
    if (c) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(c->err, sizeof(c->err), fmt, ap);
        va_end(ap);
    }
    return st;
}

#define CU(call)                                                                                     \
    do {                                                                                             \
        cudaError_t e_ = (call);                                                                     \
        if (e_ != cudaSuccess)                                                                       \
            return fail(ctx, RIOT_ECUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                        __LINE__);                                                                   \
    } while (0)

#define CU_B(call)                                                                                   \
    do {                                                                                             \
        cudaError_t e_ = (call);                                                                     \
        if (e_ != cudaSuccess) return bfail(b, RIOT_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

// Device memory of a context: from the caller's allocator when riot_options gave one,
// else cudaMalloc.  Returns NULL on failure.
void *ctx_malloc(riot_ctx *ctx, size_t bytes)
{
    if (ctx->dev_alloc) return ctx->dev_alloc(bytes, (void *)ctx->s, ctx->alloc_user);
    void *q = nullptr;
    if (cudaMalloc(&q, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return q;
}

void ctx_free(riot_ctx *ctx, const riot_alloc_rec &a)
{
    if (!a.p) return;
    if (ctx->dev_free) ctx->dev_free(a.p, a.bytes, (void *)ctx->s, ctx->alloc_user);
    else cudaFree(a.p);
}

template <typename T>
riot_status dalloc(riot_ctx *ctx, T **p, size_t count)
{
    *p = nullptr;
    if (count == 0) count = 1;
    const size_t bytes = count * sizeof(T);
    void *q = ctx_malloc(ctx, bytes);
    if (!q) return fail(ctx, RIOT_ENOMEM, "device allocation of %zu bytes failed", bytes);
    if (((uintptr_t)q & 255) != 0) {
        ctx_free(ctx, {q, bytes});
        return fail(ctx, RIOT_EINVAL, "the device allocator returned a pointer not aligned to 256 bytes");
    }
    ctx->allocs.push_back({q, bytes});
    *p = (T *)q;
    return RIOT_OK;
}

#define TRY(x)                          \
    do {                                \
        riot_status st_ = (x);          \
        if (st_ != RIOT_OK) return st_; \
    } while (0)

size_t real_size(const riot_ctx *c) { return c->prec == RIOT_PREC_FP64 ? sizeof(double) : sizeof(float); }
char real_tag(const riot_ctx *c) { return c->prec == RIOT_PREC_FP64 ? 'd' : 'f'; }

// Periodic Gaussian square-root kernel, unit-variance normalised, as a band.
void build_band(int n, double ell, std::vector<double> &band, int &hl, int &hh)
{
    std::vector<double> row(n, 0.0);
    const int reach = (int)ceil(40.0 * ell / n) + 1;
    for (int d = 0; d < n; ++d) {
        double s = 0.0;
        for (int j = -reach; j <= reach; ++j) {
            const double z = (double)d + (double)j * n;
            s += exp(-z * z / (ell * ell));
        }
        row[d] = s;
    }
    double ss = 0.0;
    for (int d = 0; d < n; ++d) ss += row[d] * row[d];
    const double alpha = 1.0 / sqrt(ss);
    for (int d = 0; d < n; ++d) row[d] *= alpha;
    int h = 0;
    for (int d = 1; d <= n / 2; ++d)
        if (fabs(row[d]) > 1e-18 * row[0]) h = d;
    if (2 * h + 1 >= n) {
        hl = (n - 1) / 2;
        hh = n / 2;
    } else {
        hl = hh = h;
    }
    band.assign(hl + hh + 1, 0.0);
    for (int d = -hl; d <= hh; ++d) band[d + hl] = row[((d % n) + n) % n];
}

void ev_mark(riot_ctx *c, int phase)
{
    if (c->nev < 32) {
        cudaEventRecord(c->ev[c->nev], c->s);
        c->ev_phase[c->nev] = phase;
        ++c->nev;
    }
}

riot_status hvp(riot_ctx *ctx, const void *W, void *Y, int64_t ld, int ncols, int add_identity)
{
    if (ctx->model == RIOT_MODEL_ADVDIFF) {
        CU(adv_hvp(ctx->a, ctx->prec == RIOT_PREC_FP64, W, Y, ld, ncols, add_identity, ctx->rscr, ctx->s));
        return RIOT_OK;
    }
    const size_t rs = real_size(ctx);
    for (int c0 = 0; c0 < ncols; c0 += ctx->kmax) {
        const int nc = (ncols - c0 < ctx->kmax) ? ncols - c0 : ctx->kmax;
        const char *w = (const char *)W + (size_t)c0 * ld * rs;
        char *yv = (char *)Y + (size_t)c0 * ld * rs;
        if (ctx->prec == RIOT_PREC_FP64)
            CU(l96_hvp_launch_f64(ctx->m, ctx->coef64, (const double *)w, (double *)yv, ld, nc, add_identity,
                                  (double *)ctx->rscr, 0, ctx->s));
        else if (ctx->coefw && (ctx->hvp_kernel == RIOT_HVP_WARP_PAIRS || ctx->hvp_kernel == RIOT_HVP_WARP_SHUFFLE))
            CU(l96_hvp_warp_launch(ctx->m, ctx->coefw, (const float *)w, (float *)yv, ld, nc, add_identity,
                                   (float *)ctx->rscr, ctx->errflag, ctx->s, ctx->hvp_S, ctx->wait_polls,
                                   ctx->hvp_kernel == RIOT_HVP_WARP_SHUFFLE));
        else
            CU(l96_hvp_tma_launch(ctx->m, ctx->coef32, (const float *)w, (float *)yv, ld, nc, add_identity,
                                  (float *)ctx->rscr, 0, ctx->errflag, ctx->s, ctx->hvp_P, ctx->hvp_S,
                                  ctx->wait_polls, ctx->hvp_kernel == RIOT_HVP_CTA_TWO_PER_SM));
    }
    return RIOT_OK;
}

// out = L in (transpose 0) or L^T in, ncols columns of n doubles
cudaError_t bsqrt(riot_ctx *ctx, const double *in, double *out, int transpose, int ncols)
{
    if (ctx->model == RIOT_MODEL_ADVDIFF) return adv_bsqrt(ctx->a, in, out, ncols, ctx->s);   // L symmetric
    return bsqrt_launch(ctx->m, in, out, transpose, ncols, ctx->s);
}

// Q (FP64, n x k) = orthonormal basis of Y (real, n x k): shifted CholeskyQR
// (shift 11 (n k + k (k + 1)) u ||Y||_F^2, Fukaya et al. 2020) followed by two
// unshifted CholeskyQR passes.  Each pass first scales the columns to unit
// norm (the Gram is scaled alike), which removes the spread of column norms
// that power-iteration blocks of strongly unstable windows carry.
// X (rows x k FP64, ld rows; rows = n when < 0) <- orthonormal basis of its columns:
// `shifted` shifted, equilibrated CholeskyQR passes, then two plain ones
riot_status cholqr64(riot_ctx *ctx, double *X, int k, int shifted, int info_base, int rows = -1)
{
    const int n = rows < 0 ? ctx->n : rows;
    for (int pass = 0; pass < shifted + 2; ++pass) {
        CU(gram_lower(n, k, X, 'd', n, ctx->G, k, ctx->s, ctx->gws, 8 * (size_t)ctx->kmax * ctx->kmax));
        CU(equilibrate(ctx->G, k, k, X, 'd', n, n, ctx->cvec, ctx->s));
        const double u = ldexp(1.0, -53);
        const double shift = (pass < shifted || ctx->qr_shift_all) ? 11.0 * ((double)n * k + (double)k * (k + 1)) * u : 0.0;
        CU(cholesky(ctx->G, k, k, shift, ctx->info + info_base + pass, ctx->gws, ctx->s, ctx->chol_whole_gpu));
        CU(trsm_right_lt(X, n, k, n, ctx->G, k, ctx->s, ctx->gws));
    }
    return RIOT_OK;
}

riot_status orth(riot_ctx *ctx, const void *Y, int k, int info_base)
{
    CU(convert_block(Y, real_tag(ctx), ctx->n, ctx->Q, 'd', ctx->n, ctx->n, k, ctx->s));
    // Each shifted pass divides the condition number by about
    // 1 / sqrt(11 (n k + k^2) u k); FP32 blocks carry at most ~1e8 of it,
    // FP64 blocks up to ~1e16.
    return cholqr64(ctx, ctx->Q, k, (ctx->prec == RIOT_PREC_FP64) ? 3 : 1, info_base);
}

// Mixed precision: Q32 = orthonormal basis of Y (FP32 block).  Grams come
// from the tensor cores to FP64-level accuracy (exact slice products) and are
// factorised in FP64 (the step that needs the range); the triangular solves
// run in FP32, like the block they act on.
riot_status orth32(riot_ctx *ctx, const float *Y, int k, int info_base, int passes, int shifted)
{
    const int n = ctx->n;
    CU(cudaMemcpyAsync(ctx->Q32, Y, sizeof(float) * (size_t)n * k, cudaMemcpyDeviceToDevice, ctx->s));
    for (int pass = 0; pass < passes; ++pass) {
        CU(tc_gram_f32(n, k, ctx->Q32, n, ctx->G, k, ctx->gws, ctx->errflag, ctx->s));
        CU(equilibrate(ctx->G, k, k, ctx->Q32, 'f', n, n, ctx->cvec, ctx->s));
        // The shift must exceed the Gram's error as well as the Cholesky's.  The sliced
        // tensor-core Gram truncates each value below 2^-36 of its column maximum; with
        // random signs that puts its 2-norm error near 2^-31 (k / n)^(1/2) of the unit
        // diagonal for columns of Gaussian-like entries.  The FP64 rounding term
        // 11 (n k + k (k + 1)) u stays above that only for large blocks: a floor of 2^-29
        // covers small ones (and thin proposal blocks) with margin.
        const double u = ldexp(1.0, -53);
        const double shift = (pass < shifted)
                                 ? fmax(11.0 * ((double)n * k + (double)k * (k + 1)) * u, ldexp(1.0, -29) / k)
                                 : 0.0;
        CU(cholesky(ctx->G, k, k, shift, ctx->info + info_base + pass, ctx->gws, ctx->s, ctx->chol_whole_gpu));
        CU(convert_block(ctx->G, 'd', k, ctx->L32, 'f', k, k, k, ctx->s));
        CU(put_block_inverses(ctx->L32, k, k, ctx->gws, ctx->s));
        CU(strsm_right_lt_inv(ctx->Q32, n, k, n, ctx->L32, k, ctx->s));
    }
    return RIOT_OK;
}

riot_status check_cholesky(riot_ctx *ctx, int base, int count, const char *what)
{
    int h[16] = {0};
    if (count > 16) count = 16;
    CU(cudaMemcpyAsync(h, ctx->info + base, sizeof(int) * count, cudaMemcpyDeviceToHost, ctx->s));
    CU(cudaStreamSynchronize(ctx->s));
    for (int i = 0; i < count; ++i) {
        if (h[i] < 0)
            return fail(ctx, RIOT_ETIMEOUT, "%s: a bounded wait of the cooperative Cholesky (pass %d) ran out", what,
                        i);
        if (h[i] != 0)
            return fail(ctx, RIOT_ENOTSPD, "%s: Cholesky pass %d met a non-positive pivot at column %d", what, i,
                        h[i] - 1);
    }
    return RIOT_OK;
}

// The flag of the kernels with bounded device waits (the mixed-precision Hessian
// kernel's stage copies, the tensor-core GEMMs' MMA completions): every call that
// launches them clears it first and reads it (synchronising) before it returns, so
// each call reports its own timeout and a later call is not blamed for it.
riot_status clear_timeout(riot_ctx *ctx)
{
    CU(cudaMemsetAsync(ctx->errflag, 0, sizeof(int), ctx->s));
    return RIOT_OK;
}

riot_status check_timeout(riot_ctx *ctx)
{
    int eflag = 0;
    CU(cudaMemcpyAsync(&eflag, ctx->errflag, sizeof(int), cudaMemcpyDeviceToHost, ctx->s));
    CU(cudaStreamSynchronize(ctx->s));
    if (!eflag) return RIOT_OK;
    CU(cudaMemsetAsync(ctx->errflag, 0, sizeof(int), ctx->s));
    if (eflag >= 2)
        return fail(ctx, RIOT_ETIMEOUT,
                    "a bounded device wait ran out and a bulk copy was still in flight when its CTA exited: every "
                    "result of that launch is invalid");
    return fail(ctx, RIOT_ETIMEOUT,
                "a bounded device wait ran out (Hessian kernel stage copy or tensor-core GEMM): the results of this "
                "call are invalid");
}

// ---------------------------------------------------------------------------
// Residual scratch of riot_hessian_apply_noalloc: a fixed device array that
// every GPU loading the library holds until the process exits, so that call
// never allocates.  Host code only sees a stand-in symbol; the device
// address is looked up once per device with cudaGetSymbolAddress.
// ---------------------------------------------------------------------------
constexpr size_t kNoAllocScratchBytes = (size_t)16 << 20;   // 16 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_addr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (first call per
// device looks it up; that first call must not be inside a stream capture).
cudaError_t noalloc_scratch(int dev, void **out)
{
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return cudaSuccess;
}

template <typename T>
cudaError_t up(riot_ctx *ctx, T *dst, const T *src, size_t count)
{
    return count ? cudaMemcpyAsync(dst, src, count * sizeof(T), cudaMemcpyHostToDevice, ctx->s) : cudaSuccess;
}

// FP64 and FP32 device copies of a host table
riot_status upload2(riot_ctx *ctx, const std::vector<double> &h, const double **d64, const float **d32)
{
    double *p64 = nullptr;
    float *p32 = nullptr;
    TRY(dalloc(ctx, &p64, h.size()));
    TRY(dalloc(ctx, &p32, h.size()));
    std::vector<float> f(h.begin(), h.end());
    cudaError_t e;
    if ((e = up(ctx, p64, h.data(), h.size())) != cudaSuccess || (e = up(ctx, p32, f.data(), f.size())) != cudaSuccess ||
        (e = cudaStreamSynchronize(ctx->s)) != cudaSuccess)
        return fail(ctx, RIOT_ECUDA, "table upload failed: %s", cudaGetErrorString(e));
    *d64 = p64;
    *d32 = p32;
    return RIOT_OK;
}

// Symmetric square root Z diag(sqrt(max(w, 0))) Z^T of the n x n row-major
// matrix A by cyclic Jacobi rotations (host, setup only).
void sym_sqrt_host(std::vector<double> &A, int n)
{
    std::vector<double> V((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                const double a2 = A[(size_t)i * n + j] * A[(size_t)i * n + j];
                tot += a2;
                if (i != j) off += a2;
            }
        if (off <= 1e-30 * tot) break;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                const double apq = A[(size_t)p * n + q];
                if (apq == 0.0) continue;
                const double tau = (A[(size_t)q * n + q] - A[(size_t)p * n + p]) / (2.0 * apq);
                const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                const double c = 1.0 / sqrt(1.0 + t * t), sn = t * c;
                for (int k = 0; k < n; ++k) {
                    double *r = &A[(size_t)k * n];
                    const double akp = r[p], akq = r[q];
                    r[p] = c * akp - sn * akq;
                    r[q] = sn * akp + c * akq;
                    double *v = &V[(size_t)k * n];
                    const double vkp = v[p], vkq = v[q];
                    v[p] = c * vkp - sn * vkq;
                    v[q] = sn * vkp + c * vkq;
                }
                for (int k = 0; k < n; ++k) {
                    const double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
                    A[(size_t)p * n + k] = c * apk - sn * aqk;
                    A[(size_t)q * n + k] = sn * apk + c * aqk;
                }
            }
    }
    std::vector<double> sw(n);
    for (int i = 0; i < n; ++i) {
        const double w = A[(size_t)i * n + i];
        sw[i] = w > 0.0 ? sqrt(w) : 0.0;
    }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double acc = 0.0;
            for (int k = 0; k < n; ++k) acc += V[(size_t)i * n + k] * sw[k] * V[(size_t)j * n + k];
            A[(size_t)i * n + j] = acc;
        }
}

riot_status setup_l96(riot_ctx *ctx, const riot_model_desc *model, const riot_obs_desc *obs, const riot_bcov_desc *B)
{
    const int64_t n64 = model->n;
    if (n64 < 16 || n64 > 8192) return fail(ctx, RIOT_EINVAL, "n = %lld outside [16, 8192]", (long long)n64);
    const int n = (int)n64, p = ctx->p, T = model->T;
    if (!isfinite(model->F)) return fail(ctx, RIOT_EINVAL, "bad F");
    if (B->kind != RIOT_B_GAUSS_RING || !(B->length > 0.0))
        return fail(ctx, RIOT_EINVAL, "bad B descriptor (kind %d, length %g)", B->kind, B->length);
    if (p > 0 && !obs->idx) return fail(ctx, RIOT_EINVAL, "null observation index array");
    for (int j = 0; j < p; ++j)
        if (obs->idx[j] < 0 || obs->idx[j] >= n) return fail(ctx, RIOT_EINVAL, "observation %d out of range", j);
    if (B->sigma_vec)
        for (int i = 0; i < n; ++i)
            if (!isfinite(B->sigma_vec[i])) return fail(ctx, RIOT_EINVAL, "non-finite sigma_vec[%d]", i);
    ctx->n = n;
    L96Dev &m = ctx->m;
    if (!choose_geom(n, &m.geom)) return fail(ctx, RIOT_EINVAL, "no thread layout for n = %d", n);
    m.T = T;
    m.dt = model->dt;
    m.F = model->F;
    m.p = p;

    std::vector<int> optr(T + 2, p), oslot(p), oidx(p);
    std::vector<double> rinv(p), yv(p);
    std::vector<float> rinv32(p);
    {
        int j = 0;
        for (int t = 0; t <= T + 1; ++t) {
            while (j < p && obs->step[j] < t) ++j;
            optr[t] = j;
        }
    }
    for (int j = 0; j < p; ++j) {
        oidx[j] = obs->idx[j];
        oslot[j] = m.geom.slot(obs->idx[j]);
        rinv[j] = 1.0 / (obs->sigma[j] * obs->sigma[j]);
        rinv32[j] = (float)rinv[j];
        yv[j] = obs->y[j];
    }
    std::vector<double> band;
    int hl = 0, hh = 0;
    build_band(n, B->length, band, hl, hh);
    std::vector<float> band32(band.begin(), band.end());
    std::vector<double> sig(n);
    std::vector<float> sig32(n);
    for (int i = 0; i < n; ++i) {
        sig[i] = B->sigma_vec ? B->sigma_vec[i] : B->sigma_b;
        sig32[i] = (float)sig[i];
    }
    m.band.hl = hl;
    m.band.hh = hh;

    const size_t np = (size_t)n, k = (size_t)ctx->kmax, rs = real_size(ctx);
    riot_status st;
    if ((st = dalloc(ctx, &ctx->optr, T + 2)) || (st = dalloc(ctx, &ctx->oslot, p)) || (st = dalloc(ctx, &ctx->oidx, p)) ||
        (st = dalloc(ctx, &ctx->y, p)) || (st = dalloc(ctx, &ctx->rinv64, p)) || (st = dalloc(ctx, &ctx->rinv32, p)) ||
        (st = dalloc(ctx, &ctx->band64, band.size())) || (st = dalloc(ctx, &ctx->band32, band.size())) ||
        (st = dalloc(ctx, &ctx->sig64, np)) || (st = dalloc(ctx, &ctx->sig32, np)) ||
        (st = dalloc(ctx, &ctx->traj, (T + 1) * np)) ||
        (st = dalloc(ctx, &ctx->coef64, (size_t)T * 4 * m.geom.Np + 1)) ||
        (ctx->prec == RIOT_PREC_MIXED && (st = dalloc(ctx, &ctx->coef32, (size_t)T * 4 * m.geom.Np + 1))) ||
        (st = dalloc(ctx, (char **)&ctx->rscr, (size_t)p * k * rs + 16)))
        return st;
    cudaError_t e = cudaSuccess;
    if ((e = up(ctx, ctx->optr, optr.data(), optr.size())) || (e = up(ctx, ctx->oslot, oslot.data(), oslot.size())) ||
        (e = up(ctx, ctx->oidx, oidx.data(), oidx.size())) || (e = up(ctx, ctx->y, yv.data(), yv.size())) ||
        (e = up(ctx, ctx->rinv64, rinv.data(), rinv.size())) || (e = up(ctx, ctx->rinv32, rinv32.data(), rinv32.size())) ||
        (e = up(ctx, ctx->band64, band.data(), band.size())) || (e = up(ctx, ctx->band32, band32.data(), band32.size())) ||
        (e = up(ctx, ctx->sig64, sig.data(), sig.size())) || (e = up(ctx, ctx->sig32, sig32.data(), sig32.size())) ||
        (e = cudaStreamSynchronize(ctx->s)))
        return fail(ctx, RIOT_ECUDA, "setup upload failed: %s", cudaGetErrorString(e));
    m.optr = ctx->optr;
    m.oslot = ctx->oslot;
    m.oidx = ctx->oidx;
    m.y = ctx->y;
    m.rinv64 = ctx->rinv64;
    m.rinv32 = ctx->rinv32;
    m.band64 = ctx->band64;
    m.band32 = ctx->band32;
    m.sig64 = ctx->sig64;
    m.sig32 = ctx->sig32;
    if (ctx->prec == RIOT_PREC_MIXED && warp_kernel_fits(m.geom)) {
        // tables of the warp-synchronous FP32 Hessian kernel
        std::vector<int> ostep, ostart, sslot, perm;
        l96_warp_tables(m.geom, T, optr, oslot, ostep, ostart, sslot, perm);
        int *d_ostep = nullptr, *d_ostart = nullptr, *d_sslot = nullptr, *d_perm = nullptr;
        if ((st = dalloc(ctx, &d_ostep, ostep.size())) || (st = dalloc(ctx, &d_ostart, ostart.size())) ||
            (st = dalloc(ctx, &d_sslot, sslot.size())) || (st = dalloc(ctx, &d_perm, perm.size())) ||
            (st = dalloc(ctx, &ctx->coefw, l96_coef_warp_floats4(m))))
            return st;
        if ((e = up(ctx, d_ostep, ostep.data(), ostep.size())) || (e = up(ctx, d_ostart, ostart.data(), ostart.size())) ||
            (e = up(ctx, d_sslot, sslot.data(), sslot.size())) || (e = up(ctx, d_perm, perm.data(), perm.size())) ||
            (e = cudaStreamSynchronize(ctx->s)))
            return fail(ctx, RIOT_ECUDA, "setup upload failed: %s", cudaGetErrorString(e));
        m.ostep = d_ostep;
        m.ostart = d_ostart;
        m.osslot = d_sslot;
        m.osperm = d_perm;
    }
    return RIOT_OK;
}

riot_status setup_advdiff(riot_ctx *ctx, const riot_model_desc *model, const riot_obs_desc *obs, const riot_bcov_desc *B)
{
    const riot_advdiff_desc *ad = model->advdiff;
    if (!ad) return fail(ctx, RIOT_EINVAL, "RIOT_MODEL_ADVDIFF needs model->advdiff");
    const int nx = ad->nx, ny = ad->ny, nz = ad->nz, nb = ad->nblocks, T = model->T, p = ctx->p;
    if (nx < 2 || ny < 2 || nz < 2 || nz > 32 || T < 1 || nb < 1 || nb > T)
        return fail(ctx, RIOT_EINVAL, "bad grid nx=%d ny=%d nz=%d nblocks=%d T=%d", nx, ny, nz, nb, T);
    if (!(ad->dx > 0.0) || !(ad->dy > 0.0) || !(ad->dz > 0.0) || !isfinite(ad->dx) || !isfinite(ad->dy) ||
        !isfinite(ad->dz))
        return fail(ctx, RIOT_EINVAL, "bad cell sizes");
    if (!ad->u || !ad->v || !ad->amp || !ad->kz || !ad->emis_b) return fail(ctx, RIOT_EINVAL, "null model array");
    const long long nyx = (long long)nx * ny, n = nyx * nb, ncells = nyx * nz;
    if (n > (1LL << 30) || ncells > (1LL << 30)) return fail(ctx, RIOT_EINVAL, "grid too large");
    if (model->n != n) return fail(ctx, RIOT_EINVAL, "n = %lld, expected nblocks*ny*nx = %lld", (long long)model->n, n);
    for (long long i = 0; i < nyx; ++i)
        if (!isfinite(ad->u[i])) return fail(ctx, RIOT_EINVAL, "non-finite u");
    for (long long i = 0; i < nyx + nx; ++i)
        if (!isfinite(ad->v[i])) return fail(ctx, RIOT_EINVAL, "non-finite v");
    for (int i = 0; i < nx; ++i)
        if (ad->v[i] != 0.0 || ad->v[(size_t)ny * nx + i] != 0.0) return fail(ctx, RIOT_EINVAL, "v must be 0 on the walls");
    for (int l = 0; l < nz; ++l)
        if (!(ad->amp[l] > 0.0) || !isfinite(ad->amp[l])) return fail(ctx, RIOT_EINVAL, "amp must be > 0");
    for (int l = 0; l <= nz; ++l)
        if (!(ad->kz[l] >= 0.0) || !isfinite(ad->kz[l])) return fail(ctx, RIOT_EINVAL, "kz must be >= 0");
    for (long long i = 0; i < n; ++i)
        if (!isfinite(ad->emis_b[i])) return fail(ctx, RIOT_EINVAL, "non-finite emis_b");
    if (B->kind != RIOT_B_EXP_SEPARABLE || !(B->length > 0.0) || !isfinite(B->length) || !(B->sigma_b > 0.0) ||
        !isfinite(B->sigma_b) || B->sigma_vec)
        return fail(ctx, RIOT_EINVAL, "the tracer model needs RIOT_B_EXP_SEPARABLE with length, sigma_b > 0");
    if (p > 0 && !obs->pos) return fail(ctx, RIOT_EINVAL, "null observation position array");
    ctx->n = (int)n;
    AdvDev &a = ctx->a;
    a.nx = nx;
    a.ny = ny;
    a.nz = nz;
    a.nb = nb;
    a.T = T;
    a.dt = model->dt;
    a.dx = ad->dx;
    a.dy = ad->dy;
    a.dz = ad->dz;
    a.sigma_b = B->sigma_b;
    a.n = n;
    a.ncells = ncells;
    a.p = p;

    // observations: trilinear corners and weights
    a.optr_h.assign(T + 2, p);
    {
        int j = 0;
        for (int t = 0; t <= T + 1; ++t) {
            while (j < p && obs->step[j] < t) ++j;
            a.optr_h[t] = j;
        }
    }
    std::vector<int> cell((size_t)8 * p);
    std::vector<double> w((size_t)8 * p), rinv(p), yv(p);
    for (int j = 0; j < p; ++j) {
        const double X = obs->pos[3 * j], Y = obs->pos[3 * j + 1], Z = obs->pos[3 * j + 2];
        if (obs->step[j] < 1 || !isfinite(X) || !(Y >= 0.0 && Y <= ny - 1.0) || !(Z >= 0.0 && Z <= nz - 1.0))
            return fail(ctx, RIOT_EINVAL, "observation %d: step or position out of range", j);
        const double fx = floor(X);
        long long i0 = (long long)fmod(fx, (double)nx);
        if (i0 < 0) i0 += nx;
        const int i1 = (int)((i0 + 1) % nx);
        const double wx = X - fx;
        int j0 = (int)floor(Y);
        if (j0 > ny - 2) j0 = ny - 2;
        const double wy = Y - j0;
        int l0 = (int)floor(Z);
        if (l0 > nz - 2) l0 = nz - 2;
        const double wz = Z - l0;
        int q = 0;
        for (int dl = 0; dl < 2; ++dl)
            for (int dj = 0; dj < 2; ++dj)
                for (int di = 0; di < 2; ++di, ++q) {
                    const int ii = di ? i1 : (int)i0;
                    cell[(size_t)8 * j + q] = (int)(((long long)(l0 + dl) * ny + (j0 + dj)) * nx + ii);
                    w[(size_t)8 * j + q] = (dl ? wz : 1.0 - wz) * (dj ? wy : 1.0 - wy) * (di ? wx : 1.0 - wx);
                }
        rinv[j] = 1.0 / (obs->sigma[j] * obs->sigma[j]);
        yv[j] = obs->y[j];
    }
    // prior square roots of the exponential correlations
    std::vector<double> Sx((size_t)nx * nx), Sy((size_t)ny * ny);
    for (int i = 0; i < nx; ++i)
        for (int j = 0; j < nx; ++j) {
            int d = abs(i - j);
            if (nx - d < d) d = nx - d;
            Sx[(size_t)i * nx + j] = exp(-(double)d * ad->dx / B->length);
        }
    for (int i = 0; i < ny; ++i)
        for (int j = 0; j < ny; ++j) Sy[(size_t)i * ny + j] = exp(-(double)abs(i - j) * ad->dy / B->length);
    sym_sqrt_host(Sx, nx);
    sym_sqrt_host(Sy, ny);

    std::vector<double> u(ad->u, ad->u + nyx), v(ad->v, ad->v + nyx + nx), amp(ad->amp, ad->amp + nz),
        kz(nz + 1, 0.0), Eb(ad->emis_b, ad->emis_b + n);
    for (int l = 1; l < nz; ++l) kz[l] = ad->kz[l];
    a.amp_h = amp;
    a.kz_h = kz;
    const double *rinv64 = nullptr, *w64 = nullptr;
    const float *rinv32 = nullptr, *w32 = nullptr, *Eb32 = nullptr;
    TRY(upload2(ctx, u, &a.u64, &a.u32));
    TRY(upload2(ctx, v, &a.v64, &a.v32));
    TRY(upload2(ctx, amp, &a.amp64, &a.amp32));
    TRY(upload2(ctx, kz, &a.kz64, &a.kz32));
    TRY(upload2(ctx, Sx, &a.Sx64, &a.Sx32));
    TRY(upload2(ctx, Sy, &a.Sy64, &a.Sy32));
    TRY(upload2(ctx, Eb, &a.Eb, &Eb32));
    TRY(upload2(ctx, w, &w64, &w32));
    TRY(upload2(ctx, rinv, &rinv64, &rinv32));
    a.w64 = w64;
    a.w32 = w32;
    a.rinv64 = rinv64;
    a.rinv32 = rinv32;
    ctx->rinv64 = const_cast<double *>(rinv64);
    int *cell_d = nullptr;
    TRY(dalloc(ctx, &cell_d, cell.size()));
    TRY(dalloc(ctx, &ctx->y, p));
    cudaError_t e;
    if ((e = up(ctx, cell_d, cell.data(), cell.size())) || (e = up(ctx, ctx->y, yv.data(), yv.size())))
        return fail(ctx, RIOT_ECUDA, "setup upload failed: %s", cudaGetErrorString(e));
    a.cell = cell_d;
    a.y = ctx->y;

    // workspace
    const bool fp64 = ctx->prec == RIOT_PREC_FP64;
    const size_t rs = real_size(ctx);
    a.Pmax64 = ctx->kmax < 64 ? ctx->kmax : 64;
    a.Pmax = fp64 ? a.Pmax64 : (ctx->kmax < 128 ? ctx->kmax : 128);
    const size_t P = (size_t)a.Pmax;
    // bytes per cell (per control) of the batch workspace: at least one FP64 probe
    const size_t wsb = P * rs > sizeof(double) ? P * rs : sizeof(double);
    a.Pws64 = (int)(wsb / sizeof(double));
    char *cA = nullptr, *cB = nullptr, *src = nullptr, *ebar = nullptr, *tmp = nullptr;
    TRY(dalloc(ctx, &cA, wsb * ncells));
    TRY(dalloc(ctx, &cB, wsb * ncells));
    TRY(dalloc(ctx, &src, wsb * n));
    TRY(dalloc(ctx, &ebar, wsb * n));
    TRY(dalloc(ctx, &tmp, wsb * n));
    a.cA = cA;
    a.cB = cB;
    a.src = src;
    a.ebar = ebar;
    a.tmp = tmp;
    TRY(dalloc(ctx, &a.c64A, ncells));
    TRY(dalloc(ctx, &a.c64B, ncells));
    TRY(dalloc(ctx, &a.ebar64, n));
    TRY(dalloc(ctx, &a.tmp64, (size_t)a.Pmax64 * n));
    TRY(dalloc(ctx, &a.Es64, n));
    TRY(dalloc(ctx, &a.Es32, n));
    TRY(dalloc(ctx, (char **)&ctx->rscr, P * (size_t)p * rs + 16));
    if ((e = cudaStreamSynchronize(ctx->s)) != cudaSuccess)
        return fail(ctx, RIOT_ECUDA, "setup failed: %s", cudaGetErrorString(e));
    return RIOT_OK;
}

size_t tcws_size(int n, int kmax)
{
    const size_t a = tc_sgemm_ws_floats(kmax, kmax, n), b = tc_sgemm_ws_floats(n, kmax, kmax);
    return a > b ? a : b;
}

// Outer-loop vectors and the model-independent inner-loop workspace.
riot_status setup_common(riot_ctx *ctx)
{
    ctx->tcws_floats = (ctx->prec == RIOT_PREC_MIXED) ? tcws_size(ctx->n, ctx->kmax) : 0;
    const size_t np = (size_t)ctx->n, k = (size_t)ctx->kmax, rs = real_size(ctx), p = (size_t)ctx->p;
    riot_status st;
    if ((st = dalloc(ctx, &ctx->x, np)) || (st = dalloc(ctx, &ctx->v, np)) || (st = dalloc(ctx, &ctx->g, np)) ||
        (st = dalloc(ctx, &ctx->dv, np)) || (st = dalloc(ctx, &ctx->tmp, np)) || (st = dalloc(ctx, &ctx->d, p)) ||
        (st = dalloc(ctx, &ctx->v0, np)) ||
        (st = dalloc(ctx, &ctx->xsave, np)) || (st = dalloc(ctx, &ctx->vsave, np)) ||
        (st = dalloc(ctx, &ctx->rd, p)) || (st = dalloc(ctx, &ctx->jo, 2)) ||
        (st = dalloc(ctx, (char **)&ctx->Wblk, np * k * rs)) || (st = dalloc(ctx, (char **)&ctx->Yblk, np * k * rs)) ||
        (st = dalloc(ctx, &ctx->Q, np * k)) || (st = dalloc(ctx, &ctx->U, np * k)) ||
        (ctx->prec == RIOT_PREC_MIXED &&
         ((st = dalloc(ctx, &ctx->Q32, np * k)) || (st = dalloc(ctx, &ctx->M32, k * k)) ||
          (st = dalloc(ctx, &ctx->N32, k * k)) || (st = dalloc(ctx, &ctx->L32, k * k)) ||
          (st = dalloc(ctx, &ctx->tcws, tcws_size(ctx->n, ctx->kmax))))) ||
        (st = dalloc(ctx, &ctx->G, k * k)) || (st = dalloc(ctx, &ctx->Mm, k * k)) || (st = dalloc(ctx, &ctx->Nm, k * k)) ||
        (st = dalloc(ctx, &ctx->Km, k * k)) || (st = dalloc(ctx, &ctx->Z, k * k)) || (st = dalloc(ctx, &ctx->lam, k)) ||
        (st = dalloc(ctx, &ctx->cvec, k)) ||
        (st = dalloc(ctx, &ctx->jwork,
                     jacobi_work_doubles((int)k) > eig_work_doubles((int)k) ? jacobi_work_doubles((int)k)
                                                                           : eig_work_doubles((int)k))) ||
        (st = dalloc(ctx, &ctx->gws, 8 * k * k > dinv_doubles((int)k) ? 8 * k * k : dinv_doubles((int)k))) ||
        (st = dalloc(ctx, &ctx->info, 32)) || (st = dalloc(ctx, &ctx->nrm, 4)) ||
        (st = dalloc(ctx, &ctx->errflag, 4)))
        return st;
    cudaError_t e;
    if ((e = cudaMemsetAsync(ctx->v, 0, sizeof(double) * np, ctx->s)) ||
        (e = cudaMemsetAsync(ctx->errflag, 0, sizeof(int) * 4, ctx->s)) ||
        (e = cudaMemsetAsync(ctx->x, 0, sizeof(double) * np, ctx->s)) || (e = cudaStreamSynchronize(ctx->s)))
        return fail(ctx, RIOT_ECUDA, "setup failed: %s", cudaGetErrorString(e));
    return RIOT_OK;
}

// Power-of-two scale of the FP32 Hessian products: |A w| / |w| for one
// Gaussian w (FP64 product) bounds the leading eigenvalue from below by a
// factor of order sqrt(n); the exponent keeps sqrt(n) * 16 * that ratio under
// 2^96, well inside the FP32 range, and is 0 for windows that need none.
riot_status choose_scale(riot_ctx *ctx)
{
    const int n = ctx->n;
    cudaStream_t s = ctx->s;
    CU(normal_launch(ctx->seed ^ 0x9e3779b97f4a7c15ULL, 0x5ca1eu, n, 1, n, 1, ctx->tmp, s));
    CU(l96_hvp_launch_f64(ctx->m, ctx->coef64, ctx->tmp, ctx->dv, n, 1, 0, ctx->rd, 0, s));
    CU(cudaMemsetAsync(ctx->nrm, 0, 4 * sizeof(double), s));
    CU(add_half_sq(n, ctx->tmp, ctx->nrm, s));
    CU(add_half_sq(n, ctx->dv, ctx->nrm + 1, s));
    double h[2] = {0.0, 0.0};
    CU(cudaMemcpyAsync(h, ctx->nrm, sizeof(h), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    // e = log2 of the bound.  The tangent-linear states grow like 2^(e/2) and the adjoint states
    // like 2^e: beyond 2^100 the input is scaled by 2^-a (in sigma, which also scales the L^T of
    // the output) and R^-1 by 2^-c, so that both stay below 2^100 and the products are
    // 2^-(2a + c) A.  2^-c must stay a normal FP32 number: windows beyond that need FP64.
    int a = 0, c = 0;
    if (h[0] > 0.0 && h[1] > 0.0 && isfinite(h[1])) {
        const double est = sqrt(h[1] / h[0]) * sqrt((double)n) * 16.0;
        const int e = (int)ceil(log2(est));
        const int eh = (e + 1) / 2;
        a = eh > 100 ? eh - 100 : 0;
        c = e - a > 100 ? e - a - 100 : 0;
    } else if (!isfinite(h[1])) {
        return fail(ctx, RIOT_ENONFINITE, "the FP64 Hessian product overflowed: the window is beyond any precision");
    }
    if (c > 120)
        return fail(ctx, RIOT_ENONFINITE,
                    "tangent-linear growth of this window (about 2^%d in the Hessian) is beyond the FP32 range; "
                    "use RIOT_PREC_FP64", a + c + 100);
    if (c != ctx->scale_rinv || c > 0) CU(scale_to_f32(ctx->p, ctx->rinv64, ldexp(1.0, -c), ctx->rinv32, s));
    if (a != ctx->scale_in || a > 0) CU(scale_to_f32(n, ctx->sig64, ldexp(1.0, -a), ctx->sig32, s));
    ctx->scale_rinv = c;
    ctx->scale_in = a;
    ctx->scale_exp = 2 * a + c;
    return RIOT_OK;
}

// FP32 sketch GEMMs of the mixed path: tensor cores (FP32-accurate three-term BF16
// splitting) for blocks of at least one 128 x 128 tile, SIMT otherwise.
cudaError_t sketch_gemm(riot_ctx *ctx, char ta, char tb, int m, int n, int k, const float *A, int64_t lda,
                        const float *B, int64_t ldb, float *C, int64_t ldc, float alpha = 1.f, float beta = 0.f)
{
    if (m >= 128 && n >= 128 && k >= 64)
        return tc_sgemm(ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, ctx->tcws, ctx->tcws_floats,
                        ctx->errflag, ctx->s);
    return sgemm(ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, ctx->s);
}

// ---------------------------------------------------------------------------
// Spectral preconditioner of Algorithm 3 (Section 2.2, Eq. 7).  Each factor
// acts on a block as X <- X + V_j diag(c_j) (V_j^T X): P_k applies the newest
// factor first, P_k^T and P_k^-1 the oldest first (every P'_j is symmetric).
// ---------------------------------------------------------------------------
enum { PC_P = 0, PC_PT = 1, PC_PINV = 2 };

void pc_free(riot_ctx *ctx)
{
    for (const riot_alloc_rec &a : ctx->pc_allocs) ctx_free(ctx, a);
    ctx->pc_allocs.clear();
    ctx->pcV = ctx->pcc = ctx->pci = ctx->pcT = ctx->pcB = nullptr;
    ctx->pcV32 = ctx->pcB32 = ctx->pcT32 = nullptr;
    ctx->pc_off.clear();
    ctx->pc_m.clear();
    ctx->pc_cap = ctx->pc_rot = ctx->pc_cols = ctx->rot_cols = 0;
}

template <typename T>
riot_status pc_alloc(riot_ctx *ctx, T **p, size_t count)
{
    const size_t bytes = (count ? count : 1) * sizeof(T);
    void *q = ctx_malloc(ctx, bytes);
    if (!q) return fail(ctx, RIOT_ENOMEM, "device allocation of %zu bytes for the preconditioner failed", bytes);
    ctx->pc_allocs.push_back({q, bytes});
    *p = (T *)q;
    return RIOT_OK;
}

// X (n x ncols FP64, ld n, ncols <= kmax) <- op(P_k) X
riot_status pc_apply64(riot_ctx *ctx, double *X, int ncols, int op)
{
    const int n = ctx->n, nf = (int)ctx->pc_m.size();
    for (int t = 0; t < nf; ++t) {
        const int j = (op == PC_P) ? nf - 1 - t : t;
        const int m = ctx->pc_m[j];
        const double *V = ctx->pcV + (size_t)ctx->pc_off[j] * n;
        const double *c = (op == PC_PINV ? ctx->pci : ctx->pcc) + ctx->pc_off[j];
        CU(gemm('T', 'N', m, ncols, n, 1.0, V, 'd', n, X, 'd', n, 0.0, ctx->pcT, 'd', m, ctx->s));
        CU(scale_rows(m, ncols, m, c, ctx->pcT, 1, ctx->s));
        CU(gemm('N', 'N', n, ncols, m, 1.0, V, 'd', n, ctx->pcT, 'd', m, 1.0, X, 'd', n, ctx->s));
    }
    return RIOT_OK;
}

// the same on an FP32 block with the FP32 copies of V_j (tensor-core GEMMs when large)
riot_status pc_apply32(riot_ctx *ctx, float *X, int ncols, int op)
{
    const int n = ctx->n, nf = (int)ctx->pc_m.size();
    for (int t = 0; t < nf; ++t) {
        const int j = (op == PC_P) ? nf - 1 - t : t;
        const int m = ctx->pc_m[j];
        const float *V = ctx->pcV32 + (size_t)ctx->pc_off[j] * n;
        const double *c = (op == PC_PINV ? ctx->pci : ctx->pcc) + ctx->pc_off[j];
        CU(sketch_gemm(ctx, 'T', 'N', m, ncols, n, V, n, X, n, ctx->pcT32, m));
        CU(scale_rows(m, ncols, m, c, ctx->pcT32, 0, ctx->s));
        CU(sketch_gemm(ctx, 'N', 'N', n, ncols, m, V, n, ctx->pcT32, m, X, n, 1.f, 1.f));
    }
    return RIOT_OK;
}

// Hessian of the inner loop on k columns (ld n, the context's real type): A of Eq. 4, or
// with preconditioner factors A_k = P_k^T P_k - I + P_k^T A P_k = P_k^T (I + A) P_k - I of
// Algorithm 3.  On the mixed path everything is in the 2^-scale_exp scaling of the FP32
// products.  The U block serves as scratch for P_k W (it is rewritten by rsvd_ritz).
riot_status inner_hvp(riot_ctx *ctx, const void *W, void *Y, int k)
{
    const int n = ctx->n;
    if (ctx->pc_m.empty()) return hvp(ctx, W, Y, n, k, 0);
    const bool f64 = (ctx->prec == RIOT_PREC_FP64);
    const double sc = ldexp(1.0, -ctx->scale_exp);
    void *Z = ctx->U;
    CU(cudaMemcpyAsync(Z, W, (size_t)n * k * real_size(ctx), cudaMemcpyDeviceToDevice, ctx->s));
    if (f64) TRY(pc_apply64(ctx, (double *)Z, k, PC_P));
    else TRY(pc_apply32(ctx, (float *)Z, k, PC_P));
    TRY(hvp(ctx, Z, Y, n, k, 0));
    CU(axpby_cols(n, k, n, sc, Z, 1.0, Y, f64, ctx->s));     // (I + A) P_k W
    if (f64) TRY(pc_apply64(ctx, (double *)Y, k, PC_PT));
    else TRY(pc_apply32(ctx, (float *)Y, k, PC_PT));
    CU(axpby_cols(n, k, n, -sc, W, 1.0, Y, f64, ctx->s));    // - W
    return RIOT_OK;
}

// Rotation of the sketch: W <- (I - U_k U_k^T) W with U_k the rotation basis, in column
// chunks of at most kmax (orthonormal chunks, so the chunked projection is the same
// projector).  Algorithm 3 then maps the columns by P_k^-1; that map is the identity on
// the complement of the span of every P_j V_j (P_j^T z = z there, by induction over the
// factors), so it is left out.
riot_status pc_rotate(riot_ctx *ctx, void *W, int k)
{
    const int n = ctx->n;
    const bool f64 = (ctx->prec == RIOT_PREC_FP64);
    for (int c0 = 0; c0 < ctx->rot_cols; c0 += ctx->kmax) {
        const int nc = (ctx->rot_cols - c0 < ctx->kmax) ? ctx->rot_cols - c0 : ctx->kmax;
        if (f64) {
            const double *B = ctx->pcB + (size_t)c0 * n;
            CU(gemm('T', 'N', nc, k, n, 1.0, B, 'd', n, W, 'd', n, 0.0, ctx->pcT, 'd', nc, ctx->s));
            CU(gemm('N', 'N', n, k, nc, -1.0, B, 'd', n, ctx->pcT, 'd', nc, 1.0, W, 'd', n, ctx->s));
        } else {
            const float *B = ctx->pcB32 + (size_t)c0 * n;
            CU(sketch_gemm(ctx, 'T', 'N', nc, k, n, B, n, (const float *)W, n, ctx->pcT32, nc));
            CU(sketch_gemm(ctx, 'N', 'N', n, k, nc, B, n, ctx->pcT32, nc, (float *)W, n, -1.f, 1.f));
        }
    }
    return RIOT_OK;
}

// Append P'_j = I + V ((lambda + 1)^-1/2 - 1) V^T (V: n x m FP64 on the device, ld n, orthonormal
// columns; lambda: m host values).  With rotation, P_k V (before the factor joins) is
// orthogonalised against the rotation basis and orthonormalised onto its end.  Synchronises.
riot_status pc_push(riot_ctx *ctx, const double *V, const double *lambda, int m)
{
    if (ctx->pc_cols + m > ctx->pc_cap)
        return fail(ctx, RIOT_EINVAL, "%d stored columns plus m = %d exceed max_cols = %d", ctx->pc_cols, m, ctx->pc_cap);
    const int n = ctx->n;
    cudaStream_t s = ctx->s;
    std::vector<double> c(m), ci(m);
    for (int i = 0; i < m; ++i) {
        const double lt = lambda[i] + 1.0;   // eigenvalue of I + A_k
        if (!(lt > 0.0) || !isfinite(lt))
            return fail(ctx, RIOT_ENONFINITE, "riot_precond_push: eigenvalue %d of I + A_k is %g", i, lt);
        c[i] = 1.0 / sqrt(lt) - 1.0;
        ci[i] = sqrt(lt) - 1.0;
    }
    if (ctx->pc_rot) {
        double *X = ctx->pcB + (size_t)ctx->rot_cols * n;
        CU(cudaMemcpyAsync(X, V, sizeof(double) * (size_t)n * m, cudaMemcpyDeviceToDevice, s));
        TRY(pc_apply64(ctx, X, m, PC_P));
        for (int pass = 0; pass < 2; ++pass)
            for (int c0 = 0; c0 < ctx->rot_cols; c0 += ctx->kmax) {
                const int nc = (ctx->rot_cols - c0 < ctx->kmax) ? ctx->rot_cols - c0 : ctx->kmax;
                const double *B = ctx->pcB + (size_t)c0 * n;
                CU(gemm('T', 'N', nc, m, n, 1.0, B, 'd', n, X, 'd', n, 0.0, ctx->pcT, 'd', nc, s));
                CU(gemm('N', 'N', n, m, nc, -1.0, B, 'd', n, ctx->pcT, 'd', nc, 1.0, X, 'd', n, s));
            }
        CU(cudaMemsetAsync(ctx->info, 0, sizeof(int) * 8, s));
        TRY(cholqr64(ctx, X, m, 3, 0));
        TRY(check_cholesky(ctx, 0, 5, "riot_precond_push (rotation basis)"));
        if (ctx->prec == RIOT_PREC_MIXED)
            CU(convert_block(X, 'd', n, ctx->pcB32 + (size_t)ctx->rot_cols * n, 'f', n, n, m, s));
    }
    const int off = ctx->pc_cols;
    CU(cudaMemcpyAsync(ctx->pcV + (size_t)off * n, V, sizeof(double) * (size_t)n * m, cudaMemcpyDeviceToDevice, s));
    if (ctx->prec == RIOT_PREC_MIXED) CU(convert_block(V, 'd', n, ctx->pcV32 + (size_t)off * n, 'f', n, n, m, s));
    CU(cudaMemcpyAsync(ctx->pcc + off, c.data(), sizeof(double) * m, cudaMemcpyHostToDevice, s));
    CU(cudaMemcpyAsync(ctx->pci + off, ci.data(), sizeof(double) * m, cudaMemcpyHostToDevice, s));
    CU(cudaStreamSynchronize(s));   // the host coefficients go out of scope
    ctx->pc_off.push_back(off);
    ctx->pc_m.push_back(m);
    ctx->pc_cols += m;
    if (ctx->pc_rot) ctx->rot_cols += m;
    ctx->pc_dirty = 1;
    return RIOT_OK;
}

riot_status rsvd_check_args(riot_ctx *ctx, int k, int q)
{
    if (!ctx->have_traj) return fail(ctx, RIOT_ESTATE, "riot_rsvd before riot_outer_begin");
    if (k < 1 || k > ctx->kmax || k > ctx->n) return fail(ctx, RIOT_EINVAL, "k = %d outside [1, min(kmax, n)]", k);
    if (q < 0 || q > 64) return fail(ctx, RIOT_EINVAL, "q = %d outside [0, 64]", q);
    if (ctx->pc_rot && ctx->rot_cols + k > ctx->n)
        return fail(ctx, RIOT_EINVAL, "rotation: k = %d plus %d resolved directions exceed n = %d", k, ctx->rot_cols,
                    ctx->n);
    return RIOT_OK;
}

// Inner loop of Algorithm 3 in phases that queue work on ctx->s and never
// synchronise, so that a batch of windows can capture them in one graph:
// rsvd_begin (sketch), [Hessian], rsvd_power + [Hessian] per power
// iteration, rsvd_end (Q, K, eigenpairs, Ritz vectors), rsvd_collect (host
// checks), increment_queue (the adaptive increment).
riot_status rsvd_begin(riot_ctx *ctx, int k, int64_t sketch_stream, const void *Omega)
{
    const int n = ctx->n;
    CU(cudaMemsetAsync(ctx->info, 0, sizeof(int) * 32, ctx->s));
    TRY(clear_timeout(ctx));
    if (Omega)
        CU(cudaMemcpyAsync(ctx->Wblk, Omega, (size_t)n * k * real_size(ctx), cudaMemcpyDeviceToDevice, ctx->s));
    else
        CU(normal_launch(ctx->seed, (uint32_t)sketch_stream, n, k, n, ctx->prec == RIOT_PREC_FP64, ctx->Wblk, ctx->s));
    if (ctx->pc_rot && ctx->rot_cols > 0) TRY(pc_rotate(ctx, ctx->Wblk, k));
    return RIOT_OK;
}

// W = orth(Y) for the next power iteration
riot_status rsvd_power(riot_ctx *ctx, int k)
{
    const int n = ctx->n;
    if (ctx->prec == RIOT_PREC_MIXED) {
        // a power-iteration basis only has to span the block well: two shifted passes
        TRY(orth32(ctx, (const float *)ctx->Yblk, k, 0, 2, 2));
        CU(cudaMemcpyAsync(ctx->Wblk, ctx->Q32, sizeof(float) * (size_t)n * k, cudaMemcpyDeviceToDevice, ctx->s));
    } else {
        TRY(orth(ctx, ctx->Yblk, k, 0));
        CU(convert_block(ctx->Q, 'd', n, ctx->Wblk, real_tag(ctx), n, n, k, ctx->s));
    }
    return RIOT_OK;
}

// Q = orth(Y), K, K = Z Lambda Z^T, U = Q Z.  with_eig = false stops before
// the eigensolver (rsvd_eig / rsvd_ritz then finish the window).
riot_status rsvd_eig(riot_ctx *ctx, int k)
{
    if (ctx->eig_method == RIOT_EIG_JACOBI)
        CU(jacobi_eig(ctx->Km, k, ctx->lam, ctx->Z, ctx->jwork, ctx->info + 12, ctx->s));
    else
        CU(tridiag_eig(ctx->Km, k, ctx->lam, ctx->Z, ctx->jwork, ctx->info + 12, ctx->s,
                       ctx->prec == RIOT_PREC_MIXED, ctx->prec == RIOT_PREC_MIXED ? ctx->errflag : nullptr));
    if (ctx->scale_exp) CU(scal(k, ldexp(1.0, ctx->scale_exp), ctx->lam, ctx->s));
    return RIOT_OK;
}

riot_status rsvd_ritz(riot_ctx *ctx, int k)
{
    const int n = ctx->n;
    cudaStream_t s = ctx->s;
    if (ctx->prec == RIOT_PREC_MIXED) {
        // U = Q Z in FP32 (Y block reused as scratch), then widened
        float *Y32 = (float *)ctx->Yblk;
        CU(convert_block(ctx->Z, 'd', k, ctx->M32, 'f', k, k, k, s));
        CU(sketch_gemm(ctx, 'N', 'N', n, k, k, ctx->Q32, n, ctx->M32, k, Y32, n));
        CU(convert_block(Y32, 'f', n, ctx->U, 'd', n, n, k, s));
    } else {
        CU(gemm('N', 'N', n, k, k, 1.0, ctx->Q, 'd', n, ctx->Z, 'd', k, 0.0, ctx->U, 'd', n, s));
    }
    CU(fix_col_signs(ctx->U, n, k, n, s));
    return RIOT_OK;
}

riot_status rsvd_end(riot_ctx *ctx, int k, bool with_eig)
{
    const int n = ctx->n;
    const char tr = real_tag(ctx);
    cudaStream_t s = ctx->s;
    const bool mixed = (ctx->prec == RIOT_PREC_MIXED);
    float *W32 = (float *)ctx->Wblk, *Y32 = (float *)ctx->Yblk;
    ev_mark(ctx, 1);
    if (mixed) TRY(orth32(ctx, Y32, k, 5, 3, 2));
    else TRY(orth(ctx, ctx->Yblk, k, 5));
    ev_mark(ctx, 2);
    if (ctx->exact_rr) {
        // K = Q^T A Q
        if (mixed) CU(cudaMemcpyAsync(W32, ctx->Q32, sizeof(float) * (size_t)n * k, cudaMemcpyDeviceToDevice, s));
        else CU(convert_block(ctx->Q, 'd', n, ctx->Wblk, tr, n, n, k, s));
        ev_mark(ctx, 0);
        TRY(inner_hvp(ctx, ctx->Wblk, ctx->Yblk, k));
        ev_mark(ctx, 2);
        if (mixed) {
            CU(sketch_gemm(ctx, 'T', 'N', k, k, n, ctx->Q32, n, Y32, n, ctx->N32, k));
            CU(convert_block(ctx->N32, 'f', k, ctx->Km, 'd', k, k, k, s));
        } else {
            CU(gemm('T', 'N', k, k, n, 1.0, ctx->Q, 'd', n, ctx->Yblk, tr, n, 0.0, ctx->Km, 'd', k, s));
        }
    } else {
        // K (Q^T W) = Q^T Y  <=>  K (M M^T) = N M^T with M = Q^T W, N = Q^T Y
        if (mixed) {
            CU(sketch_gemm(ctx, 'T', 'N', k, k, n, ctx->Q32, n, W32, n, ctx->M32, k));
            CU(sketch_gemm(ctx, 'T', 'N', k, k, n, ctx->Q32, n, Y32, n, ctx->N32, k));
            CU(convert_block(ctx->M32, 'f', k, ctx->Mm, 'd', k, k, k, s));
            CU(convert_block(ctx->N32, 'f', k, ctx->Nm, 'd', k, k, k, s));
        } else {
            CU(gemm('T', 'N', k, k, n, 1.0, ctx->Q, 'd', n, ctx->Wblk, tr, n, 0.0, ctx->Mm, 'd', k, s));
            CU(gemm('T', 'N', k, k, n, 1.0, ctx->Q, 'd', n, ctx->Yblk, tr, n, 0.0, ctx->Nm, 'd', k, s));
        }
        // K's products stay in FP64 on both paths: the solve with M M^T amplifies their
        // error by its condition number (sliced tensor-core products, exact to 2^-36 of each
        // column's maximum, moved lambda_1 of the large window by 5 %)
        CU(syrk_lower(k, k, ctx->Mm, k, ctx->G, k, s));
        CU(gemm('N', 'T', k, k, k, 1.0, ctx->Nm, 'd', k, ctx->Mm, 'd', k, 0.0, ctx->Km, 'd', k, s));
        // M M^T is singular to working precision when the window's spectrum spans more than the
        // precision (A Q0 then loses Q0's trailing directions): a retry with a shift of the order
        // of the Cholesky backward error (8 k u tr) keeps the solve defined (see rsvd_retry_k)
        const double ushift = ctx->k_shift ? 8.0 * k * ldexp(1.0, -53) : 0.0;
        CU(cholesky(ctx->G, k, k, ushift, ctx->info + 10, ctx->gws, s, ctx->chol_whole_gpu));
        CU(trsm_right_lt(ctx->Km, k, k, k, ctx->G, k, s, ctx->gws));
        CU(trsm_right_l(ctx->Km, k, k, k, ctx->G, k, s, ctx->gws));
    }
    CU(symmetrize(ctx->Km, k, k, s));
    if (!with_eig) return RIOT_OK;
    ev_mark(ctx, 3);
    TRY(rsvd_eig(ctx, k));
    ev_mark(ctx, 4);
    return rsvd_ritz(ctx, k);
}

// Host-side checks of a finished riot_rsvd; synchronises ctx->s.
riot_status rsvd_collect(riot_ctx *ctx, int k, double *lambda_out)
{
    cudaStream_t s = ctx->s;
    // a bounded wait that ran out invalidates everything after it: report it first
    TRY(check_timeout(ctx));
    TRY(check_cholesky(ctx, 0, 11, "riot_rsvd"));
    int jinfo[2] = {0, 0};
    CU(cudaMemcpyAsync(jinfo, ctx->info + 12, sizeof(jinfo), cudaMemcpyDeviceToHost, s));
    if (lambda_out) CU(cudaMemcpyAsync(lambda_out, ctx->lam, sizeof(double) * k, cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    if (ctx->eig_method == RIOT_EIG_JACOBI && jinfo[0] < 0)
        return fail(ctx, RIOT_ENOCONV, "Jacobi did not converge in %d sweeps", -jinfo[0]);
    if (ctx->eig_method == RIOT_EIG_TRIDIAG && (jinfo[0] != 0 || jinfo[1] != 0))
        return fail(ctx, RIOT_ENOCONV, "orthonormalisation of the tridiagonal eigenvectors failed");
    ctx->jacobi_sweeps = (ctx->eig_method == RIOT_EIG_JACOBI) ? jinfo[0] : 0;
    ctx->have_rsvd = 1;
    ctx->k_last = k;
    return RIOT_OK;
}

// When the unshifted Cholesky of the K normal equations failed (info[10]), redo the end of the
// inner loop with the shifted solve; the blocks Q0 (W) and Y are unchanged by rsvd_end.
// When inverse iteration met eigenvalues so close that its vectors came out dependent
// (the CholeskyQR of the eigenvectors of T failed), redo this call's eigendecomposition of
// the unchanged K with the Jacobi method, then the Ritz vectors.
riot_status rsvd_retry_eig(riot_ctx *ctx, int k, double *lambda_out, riot_status st)
{
    if (st != RIOT_ENOCONV || ctx->eig_method != RIOT_EIG_TRIDIAG) return st;
    ctx->eig_method = RIOT_EIG_JACOBI;
    riot_status st2 = rsvd_eig(ctx, k);
    if (st2 == RIOT_OK) st2 = rsvd_ritz(ctx, k);
    if (st2 == RIOT_OK) st2 = rsvd_collect(ctx, k, lambda_out);
    ctx->eig_method = RIOT_EIG_TRIDIAG;
    return st2;
}

riot_status rsvd_retry_k(riot_ctx *ctx, int k, double *lambda_out, riot_status st)
{
    if (st == RIOT_ENOCONV) return rsvd_retry_eig(ctx, k, lambda_out, st);
    if (st != RIOT_ENOTSPD) return st;
    int i10 = 0;
    CU(cudaMemcpyAsync(&i10, ctx->info + 10, sizeof(int), cudaMemcpyDeviceToHost, ctx->s));
    CU(cudaStreamSynchronize(ctx->s));
    if (i10 == 0) return st;
    ctx->k_shift = 1;
    riot_status st2 = rsvd_end(ctx, k, true);
    ctx->k_shift = 0;
    if (st2 != RIOT_OK) return st2;
    return rsvd_retry_eig(ctx, k, lambda_out, rsvd_collect(ctx, k, lambda_out));
}

// Adaptive increment (queued, no synchronisation): dv, v += dv, x += L dv.
riot_status increment_queue(riot_ctx *ctx, int k)
{
    const int n = ctx->n;
    cudaStream_t s = ctx->s;
    // c = U^T g; scale by the adaptive rule; dv = U c (- g for LRU)
    CU(gemm('T', 'N', k, 1, n, 1.0, ctx->U, 'd', n, ctx->g, 'd', n, 0.0, ctx->cvec, 'd', k, s));
    // FP32 products determine Ritz values only down to about 2^-24 lambda_1 (their rounding,
    // carried by the leading growth of the window): on the mixed path smaller pairs are not
    // retained.  The FP64 path retains all k (Algorithm 3); the deflated eigendecomposition
    // has already applied the rule level by level.
    const double floor = (ctx->prec == RIOT_PREC_MIXED && !ctx->deflated) ? ldexp(1.0, -24) : -1.0;
    CU(increment_coef(ctx->lam, k, ctx->cvec, ctx->info + 14, floor, s));
    CU(gemm('N', 'N', n, 1, k, 1.0, ctx->U, 'd', n, ctx->cvec, 'd', k, 0.0, ctx->dv, 'd', n, s));
    CU(add_if_flag(ctx->info + 14, 1, n, -1.0, ctx->g, ctx->dv, s));
    // preconditioned loop: dv = P_k dw in the control variable of x = x_b + L v
    if (!ctx->pc_m.empty()) TRY(pc_apply64(ctx, ctx->dv, 1, PC_P));
    CU(axpby(n, 1.0, ctx->dv, 1.0, ctx->v, s));
    CU(bsqrt(ctx, ctx->dv, ctx->tmp, 0, 1));
    CU(axpby(n, 1.0, ctx->tmp, 1.0, ctx->x, s));
    return RIOT_OK;
}

riot_status bfail(riot_batch *b, riot_status st, const char *fmt, ...)
{
    if (b) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(b->err, sizeof(b->err), fmt, ap);
        va_end(ap);
    }
    return st;
}

// Queue one inner loop (Algorithm 3: sketch, Y = A Omega, q power
// iterations, Q, K, eigenpairs, Ritz vectors, increment) of every window of
// the batch: per-window work on the window's branch stream, the Hessian
// products of all windows in one persistent launch on the main stream, the
// eigensolvers (cooperative, all SMs) one after another on the main stream.
riot_status batch_enqueue(riot_batch *b, int64_t sketch_stream)
{
    const int nw = (int)b->ctx.size();
    std::vector<cudaStream_t> saved(nw);
    for (int w = 0; w < nw; ++w) {
        saved[w] = b->ctx[w]->s;
        b->ctx[w]->s = b->ws[w];
        b->ctx[w]->nev = 32;   // no phase events inside a batch
        b->ctx[w]->chol_whole_gpu = false;
    }
    riot_status st = RIOT_OK;
    cudaError_t e = cudaSuccess;
    auto fork = [&]() {
        if ((e = cudaEventRecord(b->fork, b->main)) != cudaSuccess) return false;
        for (int w = 0; w < nw; ++w)
            if ((e = cudaStreamWaitEvent(b->ws[w], b->fork, 0)) != cudaSuccess) return false;
        return true;
    };
    auto join = [&]() {
        for (int w = 0; w < nw; ++w) {
            if ((e = cudaEventRecord(b->join[w], b->ws[w])) != cudaSuccess) return false;
            if ((e = cudaStreamWaitEvent(b->main, b->join[w], 0)) != cudaSuccess) return false;
        }
        return true;
    };
    do {
        if (!fork()) break;
        for (int w = 0; w < nw && st == RIOT_OK; ++w) {
            riot_ctx *c = b->ctx[w];
            if ((e = cudaMemcpyAsync(c->xsave, c->x, sizeof(double) * c->n, cudaMemcpyDeviceToDevice, c->s)) ||
                (e = cudaMemcpyAsync(c->vsave, c->v, sizeof(double) * c->n, cudaMemcpyDeviceToDevice, c->s)))
                break;
            st = rsvd_begin(c, b->k[w], sketch_stream, nullptr);
        }
        if (e != cudaSuccess) break;
        if (st != RIOT_OK || !join()) break;
        if ((e = hvp_batch_launch(b->plan, b->main)) != cudaSuccess) break;
        for (int it = 0; it < b->q && st == RIOT_OK && e == cudaSuccess; ++it) {
            if (!fork()) break;
            for (int w = 0; w < nw && st == RIOT_OK; ++w) st = rsvd_power(b->ctx[w], b->k[w]);
            if (st != RIOT_OK || !join()) break;
            e = hvp_batch_launch(b->plan, b->main);
        }
        if (st != RIOT_OK || e != cudaSuccess) break;
        if (!fork()) break;
        for (int w = 0; w < nw && st == RIOT_OK; ++w) st = rsvd_end(b->ctx[w], b->k[w], false);
        if (st != RIOT_OK || !join()) break;
        for (int w = 0; w < nw && st == RIOT_OK; ++w) {
            b->ctx[w]->s = b->main;
            st = rsvd_eig(b->ctx[w], b->k[w]);
            b->ctx[w]->s = b->ws[w];
        }
        if (st != RIOT_OK || !fork()) break;
        for (int w = 0; w < nw && st == RIOT_OK; ++w) {
            st = rsvd_ritz(b->ctx[w], b->k[w]);
            if (st == RIOT_OK) st = increment_queue(b->ctx[w], b->k[w]);
        }
        if (st != RIOT_OK) break;
        join();
    } while (0);
    for (int w = 0; w < nw; ++w) {
        b->ctx[w]->s = saved[w];
        b->ctx[w]->chol_whole_gpu = true;
    }
    if (st != RIOT_OK) return bfail(b, st, "batch: %s", "a window's inner-loop step failed (see its context)");
    if (e != cudaSuccess) return bfail(b, RIOT_ECUDA, "batch: %s", cudaGetErrorString(e));
    return RIOT_OK;
}

void batch_drop_graph(riot_batch *b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    b->graph_sketch = -1;
}

}  // namespace

extern "C" {

const char *riot_status_string(riot_status s)
{
    switch (s) {
    case RIOT_OK: return "ok";
    case RIOT_EINVAL: return "invalid argument";
    case RIOT_ENOMEM: return "out of device memory";
    case RIOT_ECUDA: return "CUDA error";
    case RIOT_ENOTSPD: return "matrix not positive definite";
    case RIOT_ETIMEOUT: return "device wait timed out";
    case RIOT_ESTATE: return "call out of order";
    case RIOT_ENOCONV: return "eigensolver did not converge";
    case RIOT_ENONFINITE: return "non-finite value";
    }
    return "unknown status";
}

const char *riot_last_error(const riot_ctx *ctx) { return ctx ? ctx->err : "no context"; }

uint64_t riot_kernel_launches(void) { return (uint64_t)launches_total(); }

void riot_destroy(riot_ctx *ctx)
{
    if (!ctx) return;
    cudaSetDevice(ctx->dev);
    if (ctx->s) cudaStreamSynchronize(ctx->s);
    pc_free(ctx);
    for (const riot_alloc_rec &a : ctx->allocs) ctx_free(ctx, a);
    for (int i = 0; i < 32; ++i)
        if (ctx->ev[i]) cudaEventDestroy(ctx->ev[i]);
    delete ctx;
}

riot_status riot_setup(riot_ctx **out, const riot_model_desc *model, const riot_obs_desc *obs, const riot_bcov_desc *B,
                       const riot_options *opt, void *cuda_stream)
{
    if (!out) return RIOT_EINVAL;
    *out = nullptr;
    if (!model || !obs || !B || !opt) return RIOT_EINVAL;
    riot_ctx *ctx = new riot_ctx();
    for (int i = 0; i < 32; ++i) ctx->ev[i] = nullptr;
    auto bail = [&](riot_status s2) {
        // keep the message readable for the caller through stderr; the context is gone
        fprintf(stderr, "riot_setup: %s\n", ctx->err);
        riot_destroy(ctx);
        return s2;
    };
    if (model->kind != RIOT_MODEL_L96 && model->kind != RIOT_MODEL_ADVDIFF)
        return bail(fail(ctx, RIOT_EINVAL, "unknown model kind %d", model->kind));
    if (opt->kmax < 1 || opt->kmax > 4096) return bail(fail(ctx, RIOT_EINVAL, "kmax = %d outside [1, 4096]", opt->kmax));
    if (opt->precision != RIOT_PREC_MIXED && opt->precision != RIOT_PREC_FP64)
        return bail(fail(ctx, RIOT_EINVAL, "unknown precision %d", opt->precision));
    const int64_t p64 = obs->p;
    if (p64 < 0 || p64 > (int64_t)1 << 30) return bail(fail(ctx, RIOT_EINVAL, "bad observation count"));
    if (p64 > 0 && (!obs->step || !obs->y || !obs->sigma))
        return bail(fail(ctx, RIOT_EINVAL, "null observation array"));
    if (model->T < 0 || !(model->dt > 0.0)) return bail(fail(ctx, RIOT_EINVAL, "bad T / dt"));
    for (int64_t j = 0; j < p64; ++j) {
        if (obs->step[j] < 0 || obs->step[j] > model->T || !(obs->sigma[j] > 0.0) || !isfinite(obs->y[j]))
            return bail(fail(ctx, RIOT_EINVAL, "observation %lld out of range", (long long)j));
        if (j > 0 && obs->step[j] < obs->step[j - 1])
            return bail(fail(ctx, RIOT_EINVAL, "observations not sorted by step at %lld", (long long)j));
    }
    ctx->eig_method = opt->eig_method;
    if (ctx->eig_method != RIOT_EIG_TRIDIAG && ctx->eig_method != RIOT_EIG_JACOBI)
        return bail(fail(ctx, RIOT_EINVAL, "unknown eig_method %d", ctx->eig_method));
    cudaGetDevice(&ctx->dev);
    ctx->s = (cudaStream_t)cuda_stream;
    ctx->prec = opt->precision;
    ctx->kmax = opt->kmax;
    ctx->exact_rr = opt->exact_rr;
    ctx->seed = opt->seed;
    if ((opt->dev_alloc == nullptr) != (opt->dev_free == nullptr))
        return bail(fail(ctx, RIOT_EINVAL, "dev_alloc and dev_free must be given together"));
    ctx->dev_alloc = opt->dev_alloc;
    ctx->dev_free = opt->dev_free;
    ctx->alloc_user = opt->alloc_user;
    ctx->model = model->kind;
    ctx->p = (int)p64;
    riot_status st = (model->kind == RIOT_MODEL_L96) ? setup_l96(ctx, model, obs, B) : setup_advdiff(ctx, model, obs, B);
    if (st != RIOT_OK) return bail(st);
    if ((st = setup_common(ctx)) != RIOT_OK) return bail(st);
    // the device address of riot_hessian_apply_noalloc's static scratch, looked up once per
    // device here so that the entry point itself never loads a module or allocates
    {
        void *scr = nullptr;
        const cudaError_t e = noalloc_scratch(ctx->dev, &scr);
        if (e != cudaSuccess)
            return bail(fail(ctx, RIOT_ECUDA, "cudaGetSymbolAddress of the static scratch failed: %s",
                             cudaGetErrorString(e)));
    }
    for (int i = 0; i < 32; ++i)
        if (cudaEventCreate(&ctx->ev[i]) != cudaSuccess) return bail(fail(ctx, RIOT_ECUDA, "cudaEventCreate failed"));
    *out = ctx;
    return RIOT_OK;
}

riot_status riot_outer_begin(riot_ctx *ctx, const double *x_dev, const double *v_dev, double *J_out)
{
    if (!ctx) return RIOT_EINVAL;
    CU(cudaSetDevice(ctx->dev));
    const int n = ctx->n;
    if (x_dev) CU(cudaMemcpyAsync(ctx->x, x_dev, sizeof(double) * n, cudaMemcpyDeviceToDevice, ctx->s));
    if (v_dev) CU(cudaMemcpyAsync(ctx->v, v_dev, sizeof(double) * n, cudaMemcpyDeviceToDevice, ctx->s));
    CU(cudaMemsetAsync(ctx->jo, 0, sizeof(double) * 2, ctx->s));
    if (ctx->model == RIOT_MODEL_ADVDIFF) {
        CU(adv_outer(ctx->a, ctx->x, ctx->d, ctx->jo, ctx->rd, ctx->g, ctx->s));
    } else {
        CU(l96_nl_launch(ctx->m, ctx->x, ctx->traj, ctx->coef32, ctx->coef64, ctx->d, ctx->jo, nullptr, ctx->s));
        if (ctx->coefw) CU(l96_coef_warp(ctx->m, ctx->coef64, ctx->coefw, ctx->s));
        // gradient b = L^T H^T R^-1 d: one FP64 adjoint integration, then g = b + v
        CU(mul(ctx->p, ctx->d, ctx->rinv64, ctx->rd, ctx->s));
        CU(l96_hvp_launch_f64(ctx->m, ctx->coef64, nullptr, ctx->g, n, 1, 0, ctx->rd, 1, ctx->s));
        if (ctx->prec == RIOT_PREC_MIXED) TRY(choose_scale(ctx));
    }
    CU(axpby(n, 1.0, ctx->v, 1.0, ctx->g, ctx->s));
    // preconditioned loop: the gradient of the problem in w (v = v_{k-1} + P_k w) is P_k^T (b + v)
    if (!ctx->pc_m.empty()) TRY(pc_apply64(ctx, ctx->g, 1, PC_PT));
    CU(add_half_sq(n, ctx->v, ctx->jo, ctx->s));
    CU(cudaMemcpyAsync(ctx->v0, ctx->v, sizeof(double) * n, cudaMemcpyDeviceToDevice, ctx->s));
    ctx->have_traj = 1;
    ctx->have_rsvd = 0;
    ctx->pc_open = 0;
    ctx->pc_dirty = 0;
    if (J_out) {
        CU(cudaMemcpyAsync(J_out, ctx->jo, sizeof(double), cudaMemcpyDeviceToHost, ctx->s));
        CU(cudaStreamSynchronize(ctx->s));
    }
    return RIOT_OK;
}

riot_status riot_hessian_apply(riot_ctx *ctx, const void *W_dev, void *Y_dev, int64_t ld, int32_t ncols,
                               int32_t add_identity)
{
    if (!ctx) return RIOT_EINVAL;
    if (!ctx->have_traj) return fail(ctx, RIOT_ESTATE, "riot_hessian_apply before riot_outer_begin");
    if (ncols < 0 || ld < ctx->n) return fail(ctx, RIOT_EINVAL, "bad ncols / ld");
    if (ncols == 0) return RIOT_OK;
    if (!W_dev || !Y_dev) return fail(ctx, RIOT_EINVAL, "null W or Y");
    CU(cudaSetDevice(ctx->dev));
    TRY(clear_timeout(ctx));
    if (!ctx->scale_exp) {
        TRY(hvp(ctx, W_dev, Y_dev, ld, ncols, add_identity));
    } else {
        TRY(hvp(ctx, W_dev, Y_dev, ld, ncols, 0));
        CU(scale_add_cols(ctx->n, ncols, ld, ldexp(1.0, ctx->scale_exp), Y_dev, add_identity ? W_dev : nullptr,
                          ctx->prec == RIOT_PREC_FP64, ctx->s));
    }
    return check_timeout(ctx);
}

riot_status riot_hessian_apply_noalloc(riot_ctx *ctx, const void *W_dev, void *Y_dev, int64_t ld, int32_t ncols,
                                       int32_t add_identity)
{
    if (!ctx) return RIOT_EINVAL;
    if (!ctx->have_traj) return fail(ctx, RIOT_ESTATE, "riot_hessian_apply_noalloc before riot_outer_begin");
    if (ncols < 0 || ld < ctx->n) return fail(ctx, RIOT_EINVAL, "bad ncols / ld");
    if (ncols == 0) return RIOT_OK;
    if (!W_dev || !Y_dev) return fail(ctx, RIOT_EINVAL, "null W or Y");
    CU(cudaSetDevice(ctx->dev));
    const size_t rs = real_size(ctx);
    const size_t per_col = (size_t)ctx->p * rs;
    if (per_col > kNoAllocScratchBytes)
        return fail(ctx, RIOT_EINVAL,
                    "riot_hessian_apply_noalloc: one column needs %zu bytes of residual scratch (%d observations), "
                    "the static array holds %zu bytes",
                    per_col, ctx->p, kNoAllocScratchBytes);
    void *scr = nullptr;
    CU(noalloc_scratch(ctx->dev, &scr));
    TRY(clear_timeout(ctx));
    size_t slice = per_col ? kNoAllocScratchBytes / per_col : (size_t)ncols;
    if (slice > (size_t)ncols) slice = (size_t)ncols;
    if (ctx->model == RIOT_MODEL_ADVDIFF && slice > (size_t)ctx->a.Pmax) slice = (size_t)ctx->a.Pmax;
    for (int c0 = 0; c0 < ncols; c0 += (int)slice) {
        const int nc = (ncols - c0 < (int)slice) ? ncols - c0 : (int)slice;
        const char *w = (const char *)W_dev + (size_t)c0 * ld * rs;
        char *yv = (char *)Y_dev + (size_t)c0 * ld * rs;
        if (ctx->model == RIOT_MODEL_ADVDIFF)
            CU(adv_hvp(ctx->a, ctx->prec == RIOT_PREC_FP64, w, yv, ld, nc, add_identity, scr, ctx->s));
        else if (ctx->prec == RIOT_PREC_FP64)
            CU(l96_hvp_launch_f64(ctx->m, ctx->coef64, (const double *)w, (double *)yv, ld, nc, add_identity,
                                  (double *)scr, 0, ctx->s));
        else {
            const int ai = ctx->scale_exp ? 0 : add_identity;
            if (ctx->coefw && (ctx->hvp_kernel == RIOT_HVP_WARP_PAIRS || ctx->hvp_kernel == RIOT_HVP_WARP_SHUFFLE))
                CU(l96_hvp_warp_launch(ctx->m, ctx->coefw, (const float *)w, (float *)yv, ld, nc, ai, (float *)scr,
                                       ctx->errflag, ctx->s, ctx->hvp_S, ctx->wait_polls,
                                       ctx->hvp_kernel == RIOT_HVP_WARP_SHUFFLE));
            else
                CU(l96_hvp_tma_launch(ctx->m, ctx->coef32, (const float *)w, (float *)yv, ld, nc, ai, (float *)scr, 0,
                                      ctx->errflag, ctx->s, ctx->hvp_P, ctx->hvp_S, ctx->wait_polls,
                                      ctx->hvp_kernel == RIOT_HVP_CTA_TWO_PER_SM));
            if (ctx->scale_exp)
                CU(scale_add_cols(ctx->n, nc, ld, ldexp(1.0, ctx->scale_exp), yv, add_identity ? w : nullptr, 0,
                                  ctx->s));
        }
    }
    return check_timeout(ctx);
}

static riot_status rsvd_run(riot_ctx *ctx, int32_t k, int32_t q, int64_t sketch_stream, const void *Omega_dev,
                            double *lambda_out)
{
    ctx->nev = 0;
    ctx->pc_ready = 0;
    ctx->pc_open = 0;
    ctx->deflated = 0;
    ev_mark(ctx, -1);
    TRY(rsvd_begin(ctx, k, sketch_stream, Omega_dev));
    ev_mark(ctx, 0);
    TRY(inner_hvp(ctx, ctx->Wblk, ctx->Yblk, k));
    for (int it = 0; it < q; ++it) {
        ev_mark(ctx, 1);
        TRY(rsvd_power(ctx, k));
        ev_mark(ctx, 0);
        TRY(inner_hvp(ctx, ctx->Wblk, ctx->Yblk, k));
    }
    TRY(rsvd_end(ctx, k, true));
    ev_mark(ctx, -2);
    TRY(rsvd_retry_k(ctx, k, lambda_out, rsvd_collect(ctx, k, lambda_out)));
    ctx->pc_open = 1;
    return RIOT_OK;
}

riot_status riot_rsvd(riot_ctx *ctx, int32_t k, int32_t q, int64_t sketch_stream, const void *Omega_dev,
                      double *lambda_out)
{
    if (!ctx) return RIOT_EINVAL;
    TRY(rsvd_check_args(ctx, k, q));
    if (ctx->pc_dirty) return fail(ctx, RIOT_ESTATE, "riot_rsvd after riot_precond_push needs riot_outer_begin first");
    CU(cudaSetDevice(ctx->dev));
    riot_status st = rsvd_run(ctx, k, q, sketch_stream, Omega_dev, lambda_out);
    if (st == RIOT_ENOTSPD && ctx->prec == RIOT_PREC_FP64) {
        // a CholeskyQR pass met a non-positive pivot: in working precision the block has fewer
        // independent columns than k (more sketch columns than the Hessian's numerical rank,
        // seen on windows with k >= 0.75 n).  Redo the inner loop with every pass shifted: the
        // basis then spans the block's range plus rounding-level directions, which give
        // eigenvalues of K near zero, as the completion of the oracle's Householder basis does.
        ctx->qr_shift_all = 1;
        st = rsvd_run(ctx, k, q, sketch_stream, Omega_dev, lambda_out);
        ctx->qr_shift_all = 0;
    }
    return st;
}

// X (n x kcols FP32, ld n) <- (I - U1 U1^T) X with U1 the first m1 columns of Ud32, in two
// passes (tensor-core FP32 GEMMs).  A Hessian product of a projected block is dominated by its
// leftover U1 components (amplified by lambda_1); one FP32 pass leaves about 2^-24 sqrt(n) of
// them, still above the smallest directions of the deflated operator, and a second pass takes
// that leftover down by the same factor again (reorthogonalisation: twice is enough).
static riot_status deflate_project(riot_ctx *ctx, float *X, int kcols, int m1)
{
    const int n = ctx->n;
    for (int pass = 0; pass < 2; ++pass) {
        CU(sketch_gemm(ctx, 'T', 'N', m1, kcols, n, ctx->Ud32, n, X, n, ctx->N32, m1));
        CU(sketch_gemm(ctx, 'N', 'N', n, kcols, m1, ctx->Ud32, n, ctx->N32, m1, X, n, -1.f, 1.f));
    }
    return RIOT_OK;
}

riot_status riot_rsvd_deflated(riot_ctx *ctx, int32_t nlevels, const int32_t *kcols, int32_t q, double rel_floor,
                               int64_t sketch_stream, double *lambda_out, int32_t *m_out)
{
    if (!ctx) return RIOT_EINVAL;
    if (ctx->prec != RIOT_PREC_MIXED) return fail(ctx, RIOT_EINVAL, "riot_rsvd_deflated: mixed-precision contexts only");
    if (!ctx->pc_m.empty()) return fail(ctx, RIOT_ESTATE, "riot_rsvd_deflated: not with the spectral preconditioner");
    if (nlevels < 1 || nlevels > 8 || !kcols) return fail(ctx, RIOT_EINVAL, "nlevels = %d outside [1, 8]", nlevels);
    TRY(rsvd_check_args(ctx, kcols[0], q));
    for (int l = 1; l < nlevels; ++l)
        if (kcols[l] < 0 || kcols[l] > ctx->kmax) return fail(ctx, RIOT_EINVAL, "kcols[%d] = %d outside [0, kmax]", l, kcols[l]);
    if (ctx->pc_dirty) return fail(ctx, RIOT_ESTATE, "riot_rsvd after riot_precond_push needs riot_outer_begin first");
    // default floor: 2^-24 of the level's largest eigenvalue, the absolute error of a level's
    // FP32 products of unit vectors
    const double fl = rel_floor > 0.0 ? rel_floor : ldexp(1.0, -24);
    CU(cudaSetDevice(ctx->dev));
    const int n = ctx->n;
    cudaStream_t s = ctx->s;
    if (!ctx->Ud64) {
        riot_status st;
        if ((st = dalloc(ctx, &ctx->Ud64, (size_t)n * ctx->kmax)) || (st = dalloc(ctx, &ctx->Ud32, (size_t)n * ctx->kmax)) ||
            (st = dalloc(ctx, &ctx->perm, (size_t)ctx->kmax))) {
            ctx->Ud64 = nullptr;
            return st;
        }
    }
    ctx->nev = 0;
    ctx->pc_ready = 0;
    ctx->pc_open = 0;
    ctx->deflated = 0;
    float *W32 = (float *)ctx->Wblk, *Y32 = (float *)ctx->Yblk;
    std::vector<double> lam_all;
    int m = 0;   // pairs kept so far: columns [0, m) of Ud64 (FP64) and Ud32 (FP32)
    ev_mark(ctx, -1);
    for (int l = 0; l < nlevels; ++l) {
        int kl = kcols[l];
        if (kl > ctx->kmax - m) kl = ctx->kmax - m;
        if (kl > n - m) kl = n - m;
        if (kl < 1) break;
        // level l: Algorithm 3 on P A P, P = I - U_m U_m^T the projector off the pairs kept so
        // far (the identity at level 0), from a sketch of its own (stream sketch_stream, its
        // top bits replaced by the level)
        CU(cudaMemsetAsync(ctx->info, 0, sizeof(int) * 32, s));
        TRY(clear_timeout(ctx));
        CU(normal_launch(ctx->seed, (uint32_t)sketch_stream ^ ((uint32_t)l << 28), n, kl, n, 0, W32, s));
        if (m > 0) TRY(deflate_project(ctx, W32, kl, m));
        ev_mark(ctx, 0);
        TRY(hvp(ctx, W32, Y32, n, kl, 0));
        if (m > 0) TRY(deflate_project(ctx, Y32, kl, m));
        for (int it = 0; it < q; ++it) {
            ev_mark(ctx, 1);
            TRY(rsvd_power(ctx, kl));
            if (m > 0) TRY(deflate_project(ctx, W32, kl, m));
            ev_mark(ctx, 0);
            TRY(hvp(ctx, W32, Y32, n, kl, 0));
            if (m > 0) TRY(deflate_project(ctx, Y32, kl, m));
        }
        TRY(rsvd_end(ctx, kl, true));
        std::vector<double> lam(kl);
        TRY(rsvd_retry_k(ctx, kl, lam.data(), rsvd_collect(ctx, kl, lam.data())));
        // a level whose largest eigenvalue is below 1, or below what even FP64 products resolve
        // (2^-53 lambda_1), adds nothing: stop
        if (l > 0 && !(lam[0] > 1.0 && lam[0] > ldexp(lam_all[0], -53))) break;
        // keep the pairs this level's FP32 products resolve: lambda >= rel_floor * its largest
        // (and > 1 after level 0, so that the adaptive rule keeps LRA where level 0 had it)
        int ml = 0;
        while (ml < kl && lam[ml] >= fl * lam[0] && (l == 0 || lam[ml] > 1.0)) ++ml;
        if (l == 0 && ml < 1) ml = 1;
        if (ml == 0) break;
        CU(cudaMemcpyAsync(ctx->Ud64 + (size_t)n * m, ctx->U, sizeof(double) * (size_t)n * ml, cudaMemcpyDeviceToDevice,
                           s));
        if (l + 1 < nlevels) CU(convert_block(ctx->U, 'd', n, ctx->Ud32 + (size_t)n * m, 'f', n, n, ml, s));
        lam_all.insert(lam_all.end(), lam.begin(), lam.begin() + ml);
        m += ml;
    }
    // ---- the pairs of every level, by decreasing eigenvalue
    std::vector<int> perm(m);
    for (int i = 0; i < m; ++i) perm[i] = i;
    std::stable_sort(perm.begin(), perm.end(), [&](int a, int b) { return lam_all[a] > lam_all[b]; });
    std::vector<double> lam_sorted(m);
    for (int i = 0; i < m; ++i) lam_sorted[i] = lam_all[perm[i]];
    CU(cudaMemcpyAsync(ctx->perm, perm.data(), sizeof(int) * m, cudaMemcpyHostToDevice, s));
    CU(cudaMemcpyAsync(ctx->lam, lam_sorted.data(), sizeof(double) * m, cudaMemcpyHostToDevice, s));
    CU(gather_cols(ctx->Ud64, n, ctx->perm, m, n, ctx->U, n, s));
    ev_mark(ctx, -2);
    CU(cudaStreamSynchronize(s));   // the host arrays go out of scope
    ctx->k_last = m;
    ctx->have_rsvd = 1;
    ctx->deflated = 1;
    ctx->pc_open = 1;
    if (lambda_out) memcpy(lambda_out, lam_sorted.data(), sizeof(double) * m);
    if (m_out) *m_out = m;
    return RIOT_OK;
}

riot_status riot_rsvd_timings(riot_ctx *ctx, double *ms_out6)
{
    if (!ctx || !ms_out6) return RIOT_EINVAL;
    CU(cudaStreamSynchronize(ctx->s));
    for (int i = 0; i < 6; ++i) ms_out6[i] = 0.0;
    for (int i = 0; i + 1 < ctx->nev; ++i) {
        float ms = 0.f;
        CU(cudaEventElapsedTime(&ms, ctx->ev[i], ctx->ev[i + 1]));
        const int ph = ctx->ev_phase[i];
        if (ph >= 0 && ph < 5) ms_out6[ph] += ms;
    }
    if (ctx->nev >= 2) {
        float ms = 0.f;
        CU(cudaEventElapsedTime(&ms, ctx->ev[0], ctx->ev[ctx->nev - 1]));
        ms_out6[5] = ms;
    }
    return RIOT_OK;
}

int32_t riot_rsvd_sweeps(const riot_ctx *ctx) { return ctx ? ctx->jacobi_sweeps : -1; }

riot_status riot_increment_pairs(riot_ctx *ctx, int32_t *m_out)
{
    if (!ctx || !m_out) return RIOT_EINVAL;
    if (!ctx->have_rsvd) return fail(ctx, RIOT_ESTATE, "riot_increment_pairs before an inner loop");
    CU(cudaSetDevice(ctx->dev));
    CU(cudaMemcpyAsync(m_out, ctx->info + 15, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->s));
    CU(cudaStreamSynchronize(ctx->s));
    return RIOT_OK;
}

riot_status riot_set_hvp_config(riot_ctx *ctx, int32_t probes_per_cta, int32_t ring_depth)
{
    if (!ctx) return RIOT_EINVAL;
    if (probes_per_cta < 0 || probes_per_cta > 64 || ring_depth < 0 || ring_depth > 8 || ring_depth == 1)
        return fail(ctx, RIOT_EINVAL, "probes_per_cta in [0, 64], ring_depth 0 or in [2, 8]");
    ctx->hvp_P = probes_per_cta;
    ctx->hvp_S = ring_depth;
    return RIOT_OK;
}

riot_status riot_set_hvp_kernel(riot_ctx *ctx, int32_t kernel)
{
    if (!ctx) return RIOT_EINVAL;
    if (kernel != RIOT_HVP_CTA_BARRIER && kernel != RIOT_HVP_WARP_PAIRS && kernel != RIOT_HVP_WARP_SHUFFLE &&
        kernel != RIOT_HVP_CTA_TWO_PER_SM)
        return fail(ctx, RIOT_EINVAL, "unknown Hessian kernel %d", kernel);
    ctx->hvp_kernel = kernel;
    return RIOT_OK;
}

riot_status riot_set_wait_limit(riot_ctx *ctx, int32_t polls)
{
    if (!ctx) return RIOT_EINVAL;
    ctx->wait_polls = polls < 0 ? -1 : polls;
    return RIOT_OK;
}

riot_status riot_quadratic_cost(riot_ctx *ctx, const double *dv_dev, double *J_out)
{
    if (!ctx || !J_out) return RIOT_EINVAL;
    if (!ctx->have_traj) return fail(ctx, RIOT_ESTATE, "riot_quadratic_cost before riot_outer_begin");
    CU(cudaSetDevice(ctx->dev));
    const int n = ctx->n;
    cudaStream_t s = ctx->s;
    double *r = nullptr;
    if (dv_dev && ctx->p > 0) {
        // r = R^-1 H M L dv: one FP64 tangent-linear integration along the stored trajectory
        r = ctx->rd;
        if (ctx->model == RIOT_MODEL_ADVDIFF) CU(adv_tl_obs(ctx->a, dv_dev, r, s));
        else CU(l96_hvp_launch_f64(ctx->m, ctx->coef64, dv_dev, nullptr, n, 1, 0, r, 2, s));
    }
    CU(cudaMemsetAsync(ctx->nrm + 2, 0, sizeof(double), s));
    CU(obs_quad_cost(ctx->p, ctx->d, r, ctx->rinv64, ctx->nrm + 2, s));
    // background term 1/2 ||v + dv||^2 with v of the last riot_outer_begin
    CU(cudaMemcpyAsync(ctx->tmp, ctx->v0, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    if (dv_dev) CU(axpby(n, 1.0, dv_dev, 1.0, ctx->tmp, s));
    CU(add_half_sq(n, ctx->tmp, ctx->nrm + 2, s));
    double h = 0.0;
    CU(cudaMemcpyAsync(&h, ctx->nrm + 2, sizeof(double), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    *J_out = h;
    return RIOT_OK;
}

riot_status riot_increment(riot_ctx *ctx, double *dv_dev, int32_t *mode_out)
{
    if (!ctx) return RIOT_EINVAL;
    if (!ctx->have_rsvd) return fail(ctx, RIOT_ESTATE, "riot_increment before riot_rsvd");
    if (ctx->pc_dirty) return fail(ctx, RIOT_ESTATE, "riot_increment after riot_precond_push needs a new inner loop");
    CU(cudaSetDevice(ctx->dev));
    TRY(increment_queue(ctx, ctx->k_last));
    ctx->pc_ready = 1;
    ctx->pc_open = 0;
    if (dv_dev) CU(cudaMemcpyAsync(dv_dev, ctx->dv, sizeof(double) * ctx->n, cudaMemcpyDeviceToDevice, ctx->s));
    if (mode_out) {
        CU(cudaMemcpyAsync(mode_out, ctx->info + 14, sizeof(int), cudaMemcpyDeviceToHost, ctx->s));
        CU(cudaStreamSynchronize(ctx->s));
    }
    return RIOT_OK;
}

riot_status riot_analysis_cov_lowrank(riot_ctx *ctx, int32_t m, double *LU_dev, double *coef_out, int32_t *mode_out)
{
    if (!ctx) return RIOT_EINVAL;
    if (!ctx->have_rsvd) return fail(ctx, RIOT_ESTATE, "riot_analysis_cov_lowrank before riot_rsvd");
    if (m < 1 || m > ctx->k_last) return fail(ctx, RIOT_EINVAL, "m = %d outside [1, k]", m);
    CU(cudaSetDevice(ctx->dev));
    cudaStream_t s = ctx->s;
    CU(cov_coef(ctx->lam, m, ctx->cvec, ctx->info + 14, s));
    if (LU_dev) CU(bsqrt(ctx, ctx->U, LU_dev, 0, m));
    if (coef_out) CU(cudaMemcpyAsync(coef_out, ctx->cvec, sizeof(double) * m, cudaMemcpyDeviceToHost, s));
    if (mode_out) CU(cudaMemcpyAsync(mode_out, ctx->info + 14, sizeof(int), cudaMemcpyDeviceToHost, s));
    if (coef_out || mode_out) CU(cudaStreamSynchronize(s));
    return RIOT_OK;
}

riot_status riot_bsqrt_apply(riot_ctx *ctx, const double *in_dev, double *out_dev, int32_t transpose, int32_t ncols)
{
    if (!ctx) return RIOT_EINVAL;
    if (ncols < 0 || (ncols > 0 && (!in_dev || !out_dev))) return fail(ctx, RIOT_EINVAL, "bad arguments");
    CU(cudaSetDevice(ctx->dev));
    CU(bsqrt(ctx, in_dev, out_dev, transpose, ncols));
    return RIOT_OK;
}

riot_status riot_get_innovation(riot_ctx *ctx, double *d_dev)
{
    if (!ctx) return RIOT_EINVAL;
    if (!ctx->have_traj) return fail(ctx, RIOT_ESTATE, "riot_get_innovation before riot_outer_begin");
    if (ctx->p > 0 && !d_dev) return fail(ctx, RIOT_EINVAL, "null d");
    CU(cudaSetDevice(ctx->dev));
    if (ctx->p > 0) CU(cudaMemcpyAsync(d_dev, ctx->d, sizeof(double) * ctx->p, cudaMemcpyDeviceToDevice, ctx->s));
    return RIOT_OK;
}

riot_status riot_get_state(riot_ctx *ctx, double *x_dev, double *v_dev, double *g_dev, double *U_dev, double *lambda_dev)
{
    if (!ctx) return RIOT_EINVAL;
    CU(cudaSetDevice(ctx->dev));
    const int n = ctx->n;
    cudaStream_t s = ctx->s;
    if (x_dev) CU(cudaMemcpyAsync(x_dev, ctx->x, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    if (v_dev) CU(cudaMemcpyAsync(v_dev, ctx->v, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    if (g_dev) CU(cudaMemcpyAsync(g_dev, ctx->g, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    if ((U_dev || lambda_dev) && !ctx->have_rsvd) return fail(ctx, RIOT_ESTATE, "no eigenpairs yet");
    if (U_dev) CU(cudaMemcpyAsync(U_dev, ctx->U, sizeof(double) * n * ctx->k_last, cudaMemcpyDeviceToDevice, s));
    if (lambda_dev) CU(cudaMemcpyAsync(lambda_dev, ctx->lam, sizeof(double) * ctx->k_last, cudaMemcpyDeviceToDevice, s));
    return RIOT_OK;
}

riot_status riot_draw_normal(uint64_t seed, int64_t stream, int64_t n, int32_t ncols, int64_t ld, int32_t is_double,
                             void *out_dev, void *cuda_stream)
{
    if (n < 0 || ncols < 0 || ld < n || (n * ncols > 0 && !out_dev)) return RIOT_EINVAL;
    cudaError_t e = normal_launch(seed, (uint32_t)stream, n, ncols, ld, is_double, out_dev, (cudaStream_t)cuda_stream);
    return e == cudaSuccess ? RIOT_OK : RIOT_ECUDA;
}

riot_status riot_symm_eig(const double *K_dev, int32_t k, double *lambda_dev, double *Z_dev, int32_t method,
                          void *cuda_stream)
{
    if (k < 1 || k > 4096 || !K_dev || !lambda_dev || !Z_dev) return RIOT_EINVAL;
    if (method != RIOT_EIG_TRIDIAG && method != RIOT_EIG_JACOBI) return RIOT_EINVAL;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const size_t nw = method == RIOT_EIG_JACOBI ? jacobi_work_doubles(k) : eig_work_doubles(k);
    double *work = nullptr, *Kc = nullptr;
    int *info = nullptr;
    if (cudaMalloc(&work, nw * sizeof(double)) != cudaSuccess) return RIOT_ENOMEM;
    if (cudaMalloc(&Kc, (size_t)k * k * sizeof(double)) != cudaSuccess || cudaMalloc(&info, 4 * sizeof(int)) != cudaSuccess) {
        cudaFree(work);
        cudaFree(Kc);
        return RIOT_ENOMEM;
    }
    riot_status st = RIOT_OK;
    cudaError_t e = cudaMemcpyAsync(Kc, K_dev, (size_t)k * k * sizeof(double), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess)
        e = (method == RIOT_EIG_JACOBI) ? jacobi_eig(Kc, k, lambda_dev, Z_dev, work, info, s)
                                        : tridiag_eig(Kc, k, lambda_dev, Z_dev, work, info, s);
    int h[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, info, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = RIOT_ECUDA;
    else if (method == RIOT_EIG_JACOBI && h[0] < 0) st = RIOT_ENOCONV;
    else if (method == RIOT_EIG_TRIDIAG && (h[0] || h[1])) st = RIOT_ENOCONV;
    cudaFree(work);
    cudaFree(Kc);
    cudaFree(info);
    return st;
}

riot_status riot_l96_forecast(int64_t n, int32_t T, double dt, double F, const double *x0_dev, double *traj_dev,
                              int32_t store_all, void *cuda_stream)
{
    if (n < 16 || n > 8192 || T < 0 || !(dt > 0.0) || !x0_dev || !traj_dev) return RIOT_EINVAL;
    L96Dev m;
    if (!choose_geom((int)n, &m.geom)) return RIOT_EINVAL;
    m.T = T;
    m.dt = dt;
    m.F = F;
    m.p = 0;
    cudaError_t e = l96_nl_launch(m, x0_dev, store_all ? traj_dev : nullptr, nullptr, nullptr, nullptr, nullptr,
                                  store_all ? nullptr : traj_dev, (cudaStream_t)cuda_stream);
    return e == cudaSuccess ? RIOT_OK : RIOT_ECUDA;
}

riot_status riot_batch_create(riot_batch **out, riot_ctx *const *ctxs, int32_t nwin, const int32_t *k, int32_t q,
                              void *cuda_stream)
{
    if (!out) return RIOT_EINVAL;
    *out = nullptr;
    if (!ctxs || !k || nwin < 1 || nwin > 4096 || q < 0 || q > 64) return RIOT_EINVAL;
    riot_batch *b = new riot_batch();
    cudaGetDevice(&b->dev);
    b->s = (cudaStream_t)cuda_stream;
    b->q = q;
    auto bail = [&](riot_status st) {
        fprintf(stderr, "riot_batch_create: %s\n", b->err);
        riot_batch_destroy(b);
        return st;
    };
    for (int w = 0; w < nwin; ++w) {
        riot_ctx *c = ctxs[w];
        if (!c) return bail(bfail(b, RIOT_EINVAL, "window %d: null context", w));
        if (c->model != RIOT_MODEL_L96 || c->prec != RIOT_PREC_MIXED || c->dev != b->dev)
            return bail(bfail(b, RIOT_EINVAL, "window %d: batches take mixed-precision Lorenz-96 contexts on one device", w));
        if (k[w] < 1 || k[w] > c->kmax || k[w] > c->n)
            return bail(bfail(b, RIOT_EINVAL, "window %d: k = %d outside [1, min(kmax, n)]", w, k[w]));
        if (c->m.geom.Tp > 512) return bail(bfail(b, RIOT_EINVAL, "window %d: n too large for the batch kernel", w));
        for (int v = 0; v < w; ++v)
            if (ctxs[v] == c) return bail(bfail(b, RIOT_EINVAL, "window %d repeats window %d", w, v));
        b->ctx.push_back(c);
        b->k.push_back(k[w]);
        cudaStream_t st = nullptr;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess)
            return bail(bfail(b, RIOT_ECUDA, "cudaStreamCreate failed"));
        b->ws.push_back(st);
        cudaEvent_t ev = nullptr;
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess)
            return bail(bfail(b, RIOT_ECUDA, "cudaEventCreate failed"));
        b->join.push_back(ev);
        riot::HvpBatchWindow hw;
        hw.m = &c->m;
        hw.coef = c->coef32;
        hw.W = (const float *)c->Wblk;
        hw.Y = (float *)c->Yblk;
        hw.ld = c->n;
        hw.ncols = k[w];
        hw.r = (float *)c->rscr;
        hw.err = c->errflag;
        b->wins.push_back(hw);
    }
    if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming) != cudaSuccess ||
        cudaStreamCreateWithFlags(&b->main, cudaStreamNonBlocking) != cudaSuccess)
        return bail(bfail(b, RIOT_ECUDA, "cudaEventCreate / cudaStreamCreate failed"));
    cudaError_t e = hvp_batch_plan(b->wins.data(), nwin, 0, 0, &b->plan);
    if (e != cudaSuccess) return bail(bfail(b, RIOT_ECUDA, "batch plan failed: %s", cudaGetErrorString(e)));
    *out = b;
    return RIOT_OK;
}

riot_status riot_batch_set_config(riot_batch *b, int32_t probes_cap, int32_t ring_depth)
{
    if (!b) return RIOT_EINVAL;
    if (probes_cap < 0 || probes_cap > 64 || ring_depth < 0 || ring_depth > 8 || ring_depth == 1)
        return bfail(b, RIOT_EINVAL, "probes_cap in [0, 64], ring_depth 0 or in [2, 8]");
    CU_B(cudaSetDevice(b->dev));
    CU_B(cudaStreamSynchronize(b->s));
    CU_B(cudaStreamSynchronize(b->main));
    batch_drop_graph(b);
    CU_B(hvp_batch_plan(b->wins.data(), (int)b->wins.size(), probes_cap, ring_depth, &b->plan));
    return RIOT_OK;
}

riot_status riot_batch_hessian_apply(riot_batch *b)
{
    if (!b) return RIOT_EINVAL;
    for (size_t w = 0; w < b->ctx.size(); ++w)
        if (!b->ctx[w]->have_traj) return bfail(b, RIOT_ESTATE, "window %zu: no riot_outer_begin yet", w);
    CU_B(cudaSetDevice(b->dev));
    CU_B(hvp_batch_launch(b->plan, b->s));
    return RIOT_OK;
}

riot_status riot_batch_autotune(riot_batch *b, int32_t *probes_cap_out, int32_t *ring_depth_out, double *ms_out)
{
    if (!b) return RIOT_EINVAL;
    for (size_t w = 0; w < b->ctx.size(); ++w)
        if (!b->ctx[w]->have_traj) return bfail(b, RIOT_ESTATE, "window %zu: no riot_outer_begin yet", w);
    CU_B(cudaSetDevice(b->dev));
    // sketches in every W block, so that the timed products see real data
    for (size_t w = 0; w < b->ctx.size(); ++w) {
        riot_ctx *c = b->ctx[w];
        CU_B(normal_launch(c->seed, 1u, c->n, b->k[w], c->n, 0, c->Wblk, b->s));
    }
    const int caps[] = {0, 32, 16, 8, 4, 2};
    const int depths[] = {4, 3, 2};
    cudaEvent_t e0, e1;
    CU_B(cudaEventCreate(&e0));
    CU_B(cudaEventCreate(&e1));
    double best = 1e300;
    int bestP = 0, bestS = 0;
    for (int P : caps)
        for (int S : depths) {
            if (hvp_batch_plan(b->wins.data(), (int)b->wins.size(), P, S, &b->plan) != cudaSuccess) {
                cudaGetLastError();
                continue;
            }
            CU_B(hvp_batch_launch(b->plan, b->s));
            CU_B(cudaEventRecord(e0, b->s));
            for (int r = 0; r < 2; ++r) CU_B(hvp_batch_launch(b->plan, b->s));
            CU_B(cudaEventRecord(e1, b->s));
            CU_B(cudaEventSynchronize(e1));
            float ms = 0.f;
            CU_B(cudaEventElapsedTime(&ms, e0, e1));
            if (ms / 2 < best) {
                best = ms / 2;
                bestP = P;
                bestS = S;
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    batch_drop_graph(b);
    CU_B(hvp_batch_plan(b->wins.data(), (int)b->wins.size(), bestP, bestS, &b->plan));
    if (probes_cap_out) *probes_cap_out = bestP;
    if (ring_depth_out) *ring_depth_out = bestS;
    if (ms_out) *ms_out = best;
    return RIOT_OK;
}

riot_status riot_batch_run(riot_batch *b, int64_t sketch_stream, int32_t use_graph, int32_t *status_out)
{
    if (!b) return RIOT_EINVAL;
    const int nw = (int)b->ctx.size();
    for (int w = 0; w < nw; ++w) {
        if (!b->ctx[w]->have_traj) return bfail(b, RIOT_ESTATE, "window %d: no riot_outer_begin yet", w);
        if (b->ctx[w]->pc_cap) return bfail(b, RIOT_EINVAL, "window %d: batches run without the spectral preconditioner", w);
    }
    CU_B(cudaSetDevice(b->dev));
    // the batch's stream follows the caller's work, and the caller's follows the batch
    CU_B(cudaEventRecord(b->done, b->s));
    CU_B(cudaStreamWaitEvent(b->main, b->done, 0));
    if (use_graph) {
        if (!b->exec || b->graph_sketch != sketch_stream) {
            batch_drop_graph(b);
            CU_B(cudaStreamBeginCapture(b->main, cudaStreamCaptureModeRelaxed));
            riot_status st = batch_enqueue(b, sketch_stream);
            cudaGraph_t g = nullptr;
            cudaError_t ce = cudaStreamEndCapture(b->main, &g);
            if (st != RIOT_OK) {
                if (g) cudaGraphDestroy(g);
                return st;
            }
            if (ce != cudaSuccess) return bfail(b, RIOT_ECUDA, "graph capture failed: %s", cudaGetErrorString(ce));
            b->graph = g;
            ce = cudaGraphInstantiate(&b->exec, g, 0);
            if (ce != cudaSuccess) {
                batch_drop_graph(b);
                return bfail(b, RIOT_ECUDA, "graph instantiation failed: %s", cudaGetErrorString(ce));
            }
            b->graph_sketch = sketch_stream;
        }
        CU_B(cudaGraphLaunch(b->exec, b->main));
    } else {
        riot_status st = batch_enqueue(b, sketch_stream);
        if (st != RIOT_OK) return st;
    }
    CU_B(cudaEventRecord(b->done, b->main));
    CU_B(cudaStreamWaitEvent(b->s, b->done, 0));
    CU_B(cudaStreamSynchronize(b->main));
    riot_status first = RIOT_OK;
    for (int w = 0; w < nw; ++w) {
        riot_status st = rsvd_collect(b->ctx[w], b->k[w], nullptr);
        if (st == RIOT_ENOTSPD) {
            // redo this window's end of the inner loop alone with the shifted K solve, then its
            // increment from the state it had before the batch ran
            riot_ctx *c = b->ctx[w];
            if (cudaMemcpyAsync(c->x, c->xsave, sizeof(double) * c->n, cudaMemcpyDeviceToDevice, c->s) != cudaSuccess ||
                cudaMemcpyAsync(c->v, c->vsave, sizeof(double) * c->n, cudaMemcpyDeviceToDevice, c->s) != cudaSuccess)
                st = RIOT_ECUDA;
            else
                st = rsvd_retry_k(c, b->k[w], nullptr, st);
            if (st == RIOT_OK) st = increment_queue(b->ctx[w], b->k[w]);
            if (st == RIOT_OK && cudaStreamSynchronize(b->ctx[w]->s) != cudaSuccess) st = RIOT_ECUDA;
        }
        if (status_out) status_out[w] = st;
        if (st != RIOT_OK && first == RIOT_OK) {
            first = st;
            bfail(b, st, "window %d: %s", w, b->ctx[w]->err);
        }
    }
    return first;
}

const char *riot_batch_last_error(const riot_batch *b) { return b ? b->err : "no batch"; }

void riot_batch_destroy(riot_batch *b)
{
    if (!b) return;
    if (b->main) cudaStreamSynchronize(b->main);
    batch_drop_graph(b);
    if (b->main) cudaStreamDestroy(b->main);
    if (b->done) cudaEventDestroy(b->done);
    hvp_batch_free(&b->plan);
    for (cudaStream_t st : b->ws) cudaStreamDestroy(st);
    for (cudaEvent_t ev : b->join) cudaEventDestroy(ev);
    if (b->fork) cudaEventDestroy(b->fork);
    delete b;
}

// ---------------------------------------------------------------------------
// Learned sketch proposal
// ---------------------------------------------------------------------------
riot_status riot_get_trajectory(riot_ctx *ctx, double *traj_dev)
{
    if (!ctx || !traj_dev) return RIOT_EINVAL;
    if (ctx->model != RIOT_MODEL_L96) return fail(ctx, RIOT_EINVAL, "riot_get_trajectory: Lorenz-96 contexts only");
    if (!ctx->have_traj) return fail(ctx, RIOT_ESTATE, "riot_get_trajectory before riot_outer_begin");
    CU(cudaSetDevice(ctx->dev));
    CU(cudaMemcpyAsync(traj_dev, ctx->traj, sizeof(double) * (size_t)(ctx->m.T + 1) * ctx->n, cudaMemcpyDeviceToDevice,
                       ctx->s));
    return RIOT_OK;
}

riot_status riot_sketchnet_create(riot_sketchnet **out, int32_t c_in, int32_t width, int32_t m_out, int32_t depth,
                                  int32_t ksize, int32_t n_max, int32_t batch_max, int32_t r_max, void *cuda_stream)
{
    if (!out) return RIOT_EINVAL;
    *out = nullptr;
    if (c_in < 1 || c_in > 256 || width < 1 || width > 1024 || m_out < 1 || m_out > 1024 || depth < 2 || depth > 8 ||
        ksize < 1 || ksize > 7 || (ksize & 1) == 0 || n_max < ksize || batch_max < 1 || r_max < 1 || r_max > n_max)
        return RIOT_EINVAL;
    riot_sketchnet *net = new riot_sketchnet();
    cudaGetDevice(&net->dev);
    net->s = (cudaStream_t)cuda_stream;
    net->net.c_in = c_in;
    net->net.width = width;
    net->net.m = m_out;
    net->net.depth = depth;
    net->net.K = ksize;
    net->net.chan[0] = c_in;
    for (int l = 1; l < depth; ++l) net->net.chan[l] = width;
    net->net.chan[depth] = m_out;
    net->n_max = n_max;
    net->b_max = batch_max;
    net->r_max = r_max;
    const size_t np = (size_t)net->net.num_params();
    const size_t n = (size_t)n_max, B = (size_t)batch_max, m = (size_t)m_out;
    const size_t wide = (size_t)(width > c_in ? width : c_in);
    auto alloc = [&](auto **p, size_t count) {
        *p = nullptr;
        if (cudaMalloc((void **)p, (count ? count : 1) * sizeof(**p)) != cudaSuccess) return false;
        net->allocs.push_back((void *)*p);
        return true;
    };
    SketchWork &w = net->w;
    if (!alloc(&net->params, np) || !alloc(&net->grad, np) || !alloc(&net->m1, np) || !alloc(&net->m2, np) ||
        !alloc(&w.Z, B * m * n) || !alloc(&w.gZ, B * m * n) || !alloc(&w.acts, (size_t)(depth - 1) * B * width * n) ||
        !alloc(&w.g0, B * wide * n) || !alloc(&w.g1, B * wide * n) || !alloc(&w.R, n * m) || !alloc(&w.XE, n * m) ||
        !alloc(&w.UtX, (size_t)r_max * m) || !alloc(&w.G, m * m) || !alloc(&w.E, m * m) || !alloc(&w.sc, 4 * B) ||
        !alloc(&net->loss, 1)) {
        riot_sketchnet_destroy(net);
        return RIOT_ENOMEM;
    }
    if (cudaMemsetAsync(net->params, 0, np * sizeof(float), net->s) != cudaSuccess ||
        cudaMemsetAsync(net->m1, 0, np * sizeof(float), net->s) != cudaSuccess ||
        cudaMemsetAsync(net->m2, 0, np * sizeof(float), net->s) != cudaSuccess ||
        cudaStreamSynchronize(net->s) != cudaSuccess) {
        riot_sketchnet_destroy(net);
        return RIOT_ECUDA;
    }
    *out = net;
    return RIOT_OK;
}

int64_t riot_sketchnet_num_params(const riot_sketchnet *net) { return net ? net->net.num_params() : -1; }

riot_status riot_sketchnet_set_params(riot_sketchnet *net, const float *params_dev)
{
    if (!net || !params_dev) return RIOT_EINVAL;
    if (cudaMemcpyAsync(net->params, params_dev, sizeof(float) * net->net.num_params(), cudaMemcpyDeviceToDevice,
                        net->s) != cudaSuccess)
        return RIOT_ECUDA;
    // a new set of weights restarts the optimiser
    if (cudaMemsetAsync(net->m1, 0, sizeof(float) * net->net.num_params(), net->s) != cudaSuccess ||
        cudaMemsetAsync(net->m2, 0, sizeof(float) * net->net.num_params(), net->s) != cudaSuccess)
        return RIOT_ECUDA;
    net->t = 0;
    return RIOT_OK;
}

riot_status riot_sketchnet_get_params(riot_sketchnet *net, float *params_dev)
{
    if (!net || !params_dev) return RIOT_EINVAL;
    return cudaMemcpyAsync(params_dev, net->params, sizeof(float) * net->net.num_params(), cudaMemcpyDeviceToDevice,
                           net->s) == cudaSuccess
               ? RIOT_OK
               : RIOT_ECUDA;
}

riot_status riot_sketchnet_forward(riot_sketchnet *net, const float *x_dev, int32_t n, int32_t batch, float *Z_dev,
                                   int32_t bf16)
{
    if (!net || !x_dev || !Z_dev || n < net->net.K || n > net->n_max || batch < 1 || batch > net->b_max)
        return RIOT_EINVAL;
    return sketchnet_forward(net->net, net->params, x_dev, n, batch, Z_dev, bf16 != 0, net->w.acts, net->s) ==
                   cudaSuccess
               ? RIOT_OK
               : RIOT_ECUDA;
}

riot_status riot_sketchnet_loss_grad(riot_sketchnet *net, const float *x_dev, const float *U_dev, int32_t r, int32_t n,
                                     int32_t batch, double mu, float *grad_dev, double *loss_out)
{
    if (!net || !x_dev || !U_dev || n < net->net.K || n > net->n_max || batch < 1 || batch > net->b_max || r < 1 ||
        r > net->r_max)
        return RIOT_EINVAL;
    float *g = grad_dev ? grad_dev : net->grad;
    if (sketchnet_loss_grad(net->net, net->params, x_dev, U_dev, r, n, batch, mu, g, net->loss, net->w, net->s) !=
        cudaSuccess)
        return RIOT_ECUDA;
    if (loss_out) {
        if (cudaMemcpyAsync(loss_out, net->loss, sizeof(double), cudaMemcpyDeviceToHost, net->s) != cudaSuccess ||
            cudaStreamSynchronize(net->s) != cudaSuccess)
            return RIOT_ECUDA;
    }
    return RIOT_OK;
}

riot_status riot_sketchnet_train_step(riot_sketchnet *net, const float *x_dev, const float *U_dev, int32_t r, int32_t n,
                                      int32_t batch, double mu, float lr, double *loss_out)
{
    riot_status st = riot_sketchnet_loss_grad(net, x_dev, U_dev, r, n, batch, mu, nullptr, nullptr);
    if (st != RIOT_OK) return st;
    net->t += 1;
    if (sketchnet_adam(net->net, net->params, net->grad, net->m1, net->m2, net->t, lr, net->s) != cudaSuccess)
        return RIOT_ECUDA;
    if (loss_out) {
        if (cudaMemcpyAsync(loss_out, net->loss, sizeof(double), cudaMemcpyDeviceToHost, net->s) != cudaSuccess ||
            cudaStreamSynchronize(net->s) != cudaSuccess)
            return RIOT_ECUDA;
    }
    return RIOT_OK;
}

riot_status riot_sketchnet_input(const double *traj_dev, int32_t T, int64_t n, int32_t c_in, float *x_dev,
                                 void *cuda_stream)
{
    if (!traj_dev || !x_dev || T < 0 || n < 1 || c_in < 1) return RIOT_EINVAL;
    double *st = nullptr;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if (cudaMalloc(&st, 2 * sizeof(double)) != cudaSuccess) return RIOT_ENOMEM;
    cudaError_t e = sketchnet_input(traj_dev, T, n, c_in, x_dev, st, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(st);
    return e == cudaSuccess ? RIOT_OK : RIOT_ECUDA;
}

void riot_sketchnet_destroy(riot_sketchnet *net)
{
    if (!net) return;
    if (net->s) cudaStreamSynchronize(net->s);
    for (void *p : net->allocs) cudaFree(p);
    delete net;
}

riot_status riot_rsvd_proposal(riot_ctx *ctx, int32_t k, int32_t q, int64_t sketch_stream, const float *P_dev, int32_t m,
                               double rho_max, double *lambda_out, double *rho_out, int32_t *used_out)
{
    if (!ctx) return RIOT_EINVAL;
    TRY(rsvd_check_args(ctx, k, q));
    if (ctx->prec != RIOT_PREC_MIXED) return fail(ctx, RIOT_EINVAL, "riot_rsvd_proposal: mixed-precision contexts only");
    if (m < 0 || m > k || (m > 0 && !P_dev)) return fail(ctx, RIOT_EINVAL, "m = %d outside [0, k] or null proposal", m);
    if (!ctx->pc_m.empty()) return fail(ctx, RIOT_ESTATE, "riot_rsvd_proposal: not with the spectral preconditioner");
    CU(cudaSetDevice(ctx->dev));
    const int n = ctx->n;
    cudaStream_t s = ctx->s;
    float *W32 = (float *)ctx->Wblk, *Y32 = (float *)ctx->Yblk;
    ctx->nev = 0;
    ctx->deflated = 0;
    ev_mark(ctx, -1);
    int used = 0;
    double rho = -1.0;
    if (m > 0) {
        CU(cudaMemsetAsync(ctx->info, 0, sizeof(int) * 32, s));
        TRY(clear_timeout(ctx));
        // the proposal, orthonormalised, then Gaussian columns for the rest of the sketch
        TRY(orth32(ctx, P_dev, m, 16, 3, 2));
        CU(cudaMemcpyAsync(W32, ctx->Q32, sizeof(float) * (size_t)n * m, cudaMemcpyDeviceToDevice, s));
        if (k > m) CU(normal_launch(ctx->seed, (uint32_t)sketch_stream, n, k - m, n, 0, W32 + (size_t)n * m, s));
        ev_mark(ctx, 0);
        TRY(hvp(ctx, W32, Y32, n, k, 0));
        // Rayleigh residual of the proposed block: rho^2 = 1 - ||Q^T A Q||_F^2 / ||A Q||_F^2
        CU(sgemm('T', 'N', m, m, n, 1.f, W32, n, Y32, n, 0.f, ctx->N32, m, s));
        CU(cudaMemsetAsync(ctx->nrm, 0, 4 * sizeof(double), s));
        CU(sumsq(ctx->N32, (size_t)m * m, ctx->nrm, s));
        CU(sumsq(Y32, (size_t)n * m, ctx->nrm + 1, s));
        double h[2] = {0, 0};
        int oi[3] = {0, 0, 0};
        CU(cudaMemcpyAsync(h, ctx->nrm, sizeof(h), cudaMemcpyDeviceToHost, s));
        CU(cudaMemcpyAsync(oi, ctx->info + 16, sizeof(oi), cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
        if (h[1] > 0.0 && isfinite(h[0]) && isfinite(h[1])) rho = sqrt(fmax(0.0, 1.0 - h[0] / h[1]));
        used = (rho >= 0.0 && rho <= rho_max && oi[0] == 0 && oi[1] == 0 && oi[2] == 0);
    }
    if (!used) {
        TRY(rsvd_begin(ctx, k, sketch_stream, nullptr));
        ev_mark(ctx, 0);
        TRY(hvp(ctx, ctx->Wblk, ctx->Yblk, n, k, 0));
    }
    for (int it = 0; it < q; ++it) {
        ev_mark(ctx, 1);
        TRY(rsvd_power(ctx, k));
        ev_mark(ctx, 0);
        TRY(hvp(ctx, ctx->Wblk, ctx->Yblk, n, k, 0));
    }
    TRY(rsvd_end(ctx, k, true));
    ev_mark(ctx, -2);
    if (rho_out) *rho_out = rho;
    if (used_out) *used_out = used;
    return rsvd_retry_k(ctx, k, lambda_out, rsvd_collect(ctx, k, lambda_out));
}

riot_status riot_tc_sgemm(char ta, char tb, int32_t m, int32_t n, int32_t k, float alpha, const float *A_dev,
                          int64_t lda, const float *B_dev, int64_t ldb, float beta, float *C_dev, int64_t ldc,
                          void *cuda_stream)
{
    if (m < 0 || n < 0 || k < 0 || (ta != 'N' && ta != 'T') || (tb != 'N' && tb != 'T')) return RIOT_EINVAL;
    if (m == 0 || n == 0) return RIOT_OK;
    if (!A_dev || !B_dev || !C_dev || ldc < m || lda < (ta == 'N' ? m : k) || ldb < (tb == 'N' ? k : n))
        return RIOT_EINVAL;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const size_t wsf = tc_sgemm_ws_floats(m, n, k);
    float *ws = nullptr;
    int *err = nullptr;
    if (wsf && cudaMalloc(&ws, wsf * sizeof(float)) != cudaSuccess) return RIOT_ENOMEM;
    if (cudaMalloc(&err, sizeof(int)) != cudaSuccess) {
        cudaFree(ws);
        return RIOT_ENOMEM;
    }
    int herr = 0;
    cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int), s);
    if (e == cudaSuccess) e = tc_sgemm(ta, tb, m, n, k, alpha, A_dev, lda, B_dev, ldb, beta, C_dev, ldc, ws, wsf, err, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(ws);
    cudaFree(err);
    if (e != cudaSuccess) return RIOT_ECUDA;
    return herr ? RIOT_ETIMEOUT : RIOT_OK;
}

// Y = A X for l <= kmax FP64 columns (ld n): the FP32 Hessian kernel and back on the mixed
// path, the power-of-two scaling of its products undone in FP64
static riot_status apply_a_block(riot_ctx *ctx, const double *X, double *Y, int l)
{
    const int n = ctx->n;
    cudaStream_t s = ctx->s;
    if (ctx->prec == RIOT_PREC_FP64) {
        TRY(hvp(ctx, X, Y, n, l, 0));
    } else {
        float *x32 = (float *)ctx->Wblk, *y32 = (float *)ctx->Yblk;
        CU(convert_block(X, 'd', n, x32, 'f', n, n, l, s));
        TRY(hvp(ctx, x32, y32, n, l, 0));
        CU(convert_block(y32, 'f', n, Y, 'd', n, n, l, s));
    }
    if (ctx->scale_exp) CU(scale_add_cols(n, l, n, ldexp(1.0, ctx->scale_exp), Y, nullptr, 1, s));
    return RIOT_OK;
}

static riot_status apply_a_vec(riot_ctx *ctx, const double *q, double *w) { return apply_a_block(ctx, q, w, 1); }

static riot_status varcg_body(riot_ctx *ctx, int32_t m, double *dv_dev, double *theta_out, int32_t *m_used)
{
    if (!ctx->have_traj) return fail(ctx, RIOT_ESTATE, "riot_varcg before riot_outer_begin");
    if (m < 1 || m > ctx->kmax) return fail(ctx, RIOT_EINVAL, "m = %d outside [1, kmax = %d]", m, ctx->kmax);
    if (!ctx->pc_m.empty()) return fail(ctx, RIOT_ESTATE, "riot_varcg: Algorithm 1 runs without the spectral preconditioner");
    CU(cudaSetDevice(ctx->dev));
    const int n = ctx->n;
    cudaStream_t s = ctx->s;
    ctx->have_rsvd = 0;   // the Lanczos basis, its Ritz vectors and values occupy the inner-loop workspace
    double *Q = ctx->Q, *r = ctx->U, *w = ctx->tmp, *h = ctx->cvec;
    double *alphas = ctx->gws, *betas_dev = ctx->gws + ctx->kmax, *rr = ctx->nrm;
    double rrh = 0.0;
    // r_0 = g, beta_0 = ||r_0||
    CU(cudaMemcpyAsync(r, ctx->g, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    CU(dot_dev(n, r, r, rr, s));
    CU(cudaMemcpyAsync(&rrh, rr, sizeof(double), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    double beta = sqrt(rrh), beta_prev = 0.0;
    std::vector<double> betas;
    int mm = 0;
    for (int i = 0; i < m; ++i) {
        if (!(beta > 0.0) || !isfinite(beta)) break;
        double *q = Q + (size_t)i * n;
        CU(normalize_by(n, r, rr, q, s));                          // q_i = r / beta
        TRY(apply_a_vec(ctx, q, w));                               // w = A q_i
        CU(dot_dev(n, q, w, alphas + i, s));                       // alpha_i = q_i^T w
        CU(lanczos_resid(n, w, q, i > 0 ? Q + (size_t)(i - 1) * n : nullptr, alphas + i, beta_prev, r, s));
        for (int pass = 0; pass < 2; ++pass) {                     // full re-orthogonalisation, twice
            CU(gemm('T', 'N', i + 1, 1, n, 1.0, Q, 'd', n, r, 'd', n, 0.0, h, 'd', i + 1, s));
            CU(gemm('N', 'N', n, 1, i + 1, -1.0, Q, 'd', n, h, 'd', i + 1, 1.0, r, 'd', n, s));
        }
        beta_prev = beta;
        CU(dot_dev(n, r, r, rr, s));
        CU(cudaMemcpyAsync(&rrh, rr, sizeof(double), cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
        beta = sqrt(rrh);
        betas.push_back(beta);
        mm = i + 1;
    }
    if (mm == 0) {
        // g = 0: the increment is zero
        if (dv_dev) CU(cudaMemsetAsync(dv_dev, 0, sizeof(double) * n, s));
        if (m_used) *m_used = 0;
        CU(cudaStreamSynchronize(s));
        return RIOT_OK;
    }
    // T_m, its eigenpairs (theta, Z), U = Q Z, dv = -U diag(1 / (1 + theta)) U^T g
    CU(cudaMemcpyAsync(betas_dev, betas.data(), sizeof(double) * mm, cudaMemcpyHostToDevice, s));
    CU(tridiag_fill(mm, alphas, betas_dev, ctx->Km, s));
    CU(tridiag_eig(ctx->Km, mm, ctx->lam, ctx->Z, ctx->jwork, ctx->info + 12, s));
    int einfo[2] = {0, 0};
    CU(cudaMemcpyAsync(einfo, ctx->info + 12, sizeof(einfo), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    if (einfo[0] || einfo[1]) {
        // close Ritz values left inverse iteration with dependent vectors: Jacobi on T_m instead
        CU(jacobi_eig(ctx->Km, mm, ctx->lam, ctx->Z, ctx->jwork, ctx->info + 12, s));
        CU(cudaMemcpyAsync(einfo, ctx->info + 12, sizeof(einfo), cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
        if (einfo[0] < 0) return fail(ctx, RIOT_ENOCONV, "riot_varcg: Jacobi on T_m did not converge");
    }
    CU(gemm('N', 'N', n, mm, mm, 1.0, Q, 'd', n, ctx->Z, 'd', mm, 0.0, ctx->U, 'd', n, s));
    CU(gemm('T', 'N', mm, 1, n, 1.0, ctx->U, 'd', n, ctx->g, 'd', n, 0.0, ctx->cvec, 'd', mm, s));
    CU(div_one_plus(mm, ctx->cvec, ctx->lam, s));
    CU(gemm('N', 'N', n, 1, mm, -1.0, ctx->U, 'd', n, ctx->cvec, 'd', mm, 0.0, ctx->dv, 'd', n, s));
    if (dv_dev) CU(cudaMemcpyAsync(dv_dev, ctx->dv, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    if (theta_out) CU(cudaMemcpyAsync(theta_out, ctx->lam, sizeof(double) * mm, cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    if (m_used) *m_used = mm;
    return RIOT_OK;
}

// Eigenpairs of the k x k matrix in Km (not modified by the tridiagonal solver) into lam, Z:
// the tridiagonal solver, and Jacobi when close eigenvalues left inverse iteration with
// dependent vectors.  Synchronises.
static riot_status small_eig(riot_ctx *ctx, int k, const char *what)
{
    cudaStream_t s = ctx->s;
    CU(tridiag_eig(ctx->Km, k, ctx->lam, ctx->Z, ctx->jwork, ctx->info + 12, s));
    int einfo[2] = {0, 0};
    CU(cudaMemcpyAsync(einfo, ctx->info + 12, sizeof(einfo), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    if (einfo[0] || einfo[1]) {
        CU(jacobi_eig(ctx->Km, k, ctx->lam, ctx->Z, ctx->jwork, ctx->info + 12, s));
        CU(cudaMemcpyAsync(einfo, ctx->info + 12, sizeof(einfo), cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
        if (einfo[0] < 0) return fail(ctx, RIOT_ENOCONV, "%s: Jacobi did not converge", what);
    }
    return RIOT_OK;
}

static riot_status varbl_body(riot_ctx *ctx, int32_t l, int32_t m, const double *B0_dev, double *dv_dev,
                              double *theta_out, int32_t *blocks_used)
{
    if (!ctx->have_traj) return fail(ctx, RIOT_ESTATE, "riot_varbl before riot_outer_begin");
    if (l < 1 || m < 1 || (int64_t)l * m > ctx->kmax || (int64_t)l * m > ctx->n)
        return fail(ctx, RIOT_EINVAL, "l = %d, m = %d: 1 <= l m <= min(kmax = %d, n = %d) required", l, m, ctx->kmax,
                    ctx->n);
    if (!B0_dev) return fail(ctx, RIOT_EINVAL, "riot_varbl: null starting block");
    if (!ctx->pc_m.empty()) return fail(ctx, RIOT_ESTATE, "riot_varbl: Algorithm 2 runs without the spectral preconditioner");
    CU(cudaSetDevice(ctx->dev));
    const int n = ctx->n;
    cudaStream_t s = ctx->s;
    ctx->have_rsvd = 0;   // the block basis and its Ritz vectors occupy the inner-loop workspace
    ctx->pc_open = 0;
    double *Q = ctx->Q, *Y = ctx->U, *H = ctx->G, *blocks = ctx->jwork;
    const int64_t ll = (int64_t)l * l;
    // Q_1 = orth(B0)
    CU(cudaMemcpyAsync(Q, B0_dev, sizeof(double) * (size_t)n * l, cudaMemcpyDeviceToDevice, s));
    CU(cudaMemsetAsync(ctx->info, 0, sizeof(int) * 8, s));
    TRY(cholqr64(ctx, Q, l, 3, 0));
    TRY(check_cholesky(ctx, 0, 5, "riot_varbl (the gradient samples are dependent)"));
    std::vector<double> hM((size_t)ll), hW((size_t)ll);
    // B0 = Q_1 W_0 with W_0 = Q_1^T B0 upper triangular: a diagonal entry far below the largest
    // means dependent samples (shifted CholeskyQR would otherwise orthonormalise rounding noise)
    CU(gemm('T', 'N', l, l, n, 1.0, Q, 'd', n, B0_dev, 'd', n, 0.0, blocks, 'd', l, s));
    CU(cudaMemcpyAsync(hW.data(), blocks, sizeof(double) * ll, cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    {
        double dmax = 0.0, dmin = INFINITY;
        for (int j = 0; j < l; ++j) {
            const double d = fabs(hW[j + (int64_t)j * l]);
            dmax = fmax(dmax, d);
            dmin = fmin(dmin, d);
        }
        if (!(dmin > 1e-12 * dmax))
            return fail(ctx, RIOT_ENOTSPD, "riot_varbl: the gradient samples are dependent (%g of the largest)",
                        dmax > 0 ? dmin / dmax : 0.0);
    }
    double scale = 0.0;
    int nb = 0;
    for (int i = 0; i < m; ++i) {
        double *Qi = Q + (size_t)i * l * n;
        double *Mi = blocks + i * ll;
        TRY(apply_a_block(ctx, Qi, Y, l));                                                   // Y_i = A Q_i
        CU(gemm('T', 'N', l, l, n, 1.0, Qi, 'd', n, Y, 'd', n, 0.0, Mi, 'd', l, s));         // M_i = Q_i^T Y_i
        nb = i + 1;
        if (i == m - 1) break;
        CU(cudaMemcpyAsync(hM.data(), Mi, sizeof(double) * ll, cudaMemcpyDeviceToHost, s));
        // r = Y_i - Q_i M_i - Q_{i-1} W_{i-1}^T, then re-orthogonalised against Q_1 .. Q_i twice
        CU(gemm('N', 'N', n, l, l, -1.0, Qi, 'd', n, Mi, 'd', l, 1.0, Y, 'd', n, s));
        if (i > 0)
            CU(gemm('N', 'T', n, l, l, -1.0, Q + (size_t)(i - 1) * l * n, 'd', n, blocks + (m + i - 1) * ll, 'd', l,
                    1.0, Y, 'd', n, s));
        const int c = (i + 1) * l;
        for (int pass = 0; pass < 2; ++pass) {
            CU(gemm('T', 'N', c, l, n, 1.0, Q, 'd', n, Y, 'd', n, 0.0, H, 'd', c, s));
            CU(gemm('N', 'N', n, l, c, -1.0, Q, 'd', n, H, 'd', c, 1.0, Y, 'd', n, s));
        }
        // Q_{i+1} W_i = r: CholeskyQR of a copy of r, then W_i = Q_{i+1}^T r (upper triangular,
        // positive diagonal: the product of the passes' factors)
        double *Qn = Q + (size_t)(i + 1) * l * n;
        double *Wi = blocks + (m + i) * ll;
        CU(cudaMemcpyAsync(Qn, Y, sizeof(double) * (size_t)n * l, cudaMemcpyDeviceToDevice, s));
        CU(cudaMemsetAsync(ctx->info, 0, sizeof(int) * 8, s));
        TRY(cholqr64(ctx, Qn, l, 3, 0));
        CU(gemm('T', 'N', l, l, n, 1.0, Qn, 'd', n, Y, 'd', n, 0.0, Wi, 'd', l, s));
        int h[5] = {0, 0, 0, 0, 0};
        CU(cudaMemcpyAsync(h, ctx->info, sizeof(h), cudaMemcpyDeviceToHost, s));
        CU(cudaMemcpyAsync(hW.data(), Wi, sizeof(double) * ll, cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
        for (int64_t e = 0; e < ll; ++e) scale = fmax(scale, fabs(hM[e]));
        bool lost = h[0] || h[1] || h[2] || h[3] || h[4];
        for (int j = 0; j < l && !lost; ++j) lost = !(fabs(hW[j + (int64_t)j * l]) > 1e-12 * scale);
        if (lost) break;   // the residual block lost rank: the block Krylov space is invariant
    }
    const int K = nb * l;
    CU(block_tridiag_fill(nb, l, m, blocks, ctx->Km, s));
    TRY(small_eig(ctx, K, "riot_varbl"));
    // U = Q Z, dv = -U diag(1 / (1 + lambda)) U^T g
    CU(gemm('N', 'N', n, K, K, 1.0, Q, 'd', n, ctx->Z, 'd', K, 0.0, ctx->U, 'd', n, s));
    CU(gemm('T', 'N', K, 1, n, 1.0, ctx->U, 'd', n, ctx->g, 'd', n, 0.0, ctx->cvec, 'd', K, s));
    CU(div_one_plus(K, ctx->cvec, ctx->lam, s));
    CU(gemm('N', 'N', n, 1, K, -1.0, ctx->U, 'd', n, ctx->cvec, 'd', K, 0.0, ctx->dv, 'd', n, s));
    if (dv_dev) CU(cudaMemcpyAsync(dv_dev, ctx->dv, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    if (theta_out) CU(cudaMemcpyAsync(theta_out, ctx->lam, sizeof(double) * K, cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    if (blocks_used) *blocks_used = nb;
    return RIOT_OK;
}

// Algorithms 1 and 2 launch the Hessian kernel (bounded waits on the mixed path) once per step:
// the wait flag is cleared before the first and read after the last
riot_status riot_varcg(riot_ctx *ctx, int32_t m, double *dv_dev, double *theta_out, int32_t *m_used)
{
    if (!ctx) return RIOT_EINVAL;
    CU(cudaSetDevice(ctx->dev));
    TRY(clear_timeout(ctx));
    const riot_status st = varcg_body(ctx, m, dv_dev, theta_out, m_used);
    const riot_status tst = check_timeout(ctx);
    return tst != RIOT_OK ? tst : st;
}

riot_status riot_varbl(riot_ctx *ctx, int32_t l, int32_t m, const double *B0_dev, double *dv_dev, double *theta_out,
                       int32_t *blocks_used)
{
    if (!ctx) return RIOT_EINVAL;
    CU(cudaSetDevice(ctx->dev));
    TRY(clear_timeout(ctx));
    const riot_status st = varbl_body(ctx, l, m, B0_dev, dv_dev, theta_out, blocks_used);
    const riot_status tst = check_timeout(ctx);
    return tst != RIOT_OK ? tst : st;
}

// ---------------------------------------------------------------------------
// RIOT-PSAS (Appendix, Algorithm 4): the randomized eigendecomposition in observation space.
// ---------------------------------------------------------------------------
static riot_status psas_alloc(riot_ctx *ctx)
{
    if (ctx->psW) return RIOT_OK;
    const size_t p = (size_t)ctx->p, pk = p * (size_t)ctx->kmax;
    riot_status st;
    if ((st = dalloc(ctx, &ctx->psW, pk)) || (st = dalloc(ctx, &ctx->psY, pk)) || (st = dalloc(ctx, &ctx->psQ, pk)) ||
        (st = dalloc(ctx, &ctx->psU, pk)) || (st = dalloc(ctx, &ctx->psF, pk)) || (st = dalloc(ctx, &ctx->psR, pk)) ||
        (st = dalloc(ctx, &ctx->psS, p)) || (st = dalloc(ctx, &ctx->psSig, p)) || (st = dalloc(ctx, &ctx->psr, p)) ||
        (st = dalloc(ctx, &ctx->psw, p)) || (st = dalloc(ctx, &ctx->psc, (size_t)ctx->kmax))) {
        ctx->psW = nullptr;
        return st;
    }
    // S = diag(1 / sigma_o) and sigma_o from R^-1 = diag(1 / sigma_o^2)
    std::vector<double> ri(p), sv(p), sg(p);
    CU(cudaMemcpyAsync(ri.data(), ctx->rinv64, sizeof(double) * p, cudaMemcpyDeviceToHost, ctx->s));
    CU(cudaStreamSynchronize(ctx->s));
    for (size_t i = 0; i < p; ++i) {
        sv[i] = sqrt(ri[i]);
        sg[i] = 1.0 / sv[i];
    }
    CU(cudaMemcpyAsync(ctx->psS, sv.data(), sizeof(double) * p, cudaMemcpyHostToDevice, ctx->s));
    CU(cudaMemcpyAsync(ctx->psSig, sg.data(), sizeof(double) * p, cudaMemcpyHostToDevice, ctx->s));
    CU(cudaStreamSynchronize(ctx->s));
    return RIOT_OK;
}

// Y = A_dual W = S H B H^T S W for m <= kmax observation-space columns (ld p), FP64 on either
// precision: the adjoint from the forcing S w and L^T, then L, the tangent linear model and
// R^-1 H, then sigma_o (S R = diag(sigma_o)).  ctx->U holds the n x m intermediate
// L^T H^T S W (Lorenz-96: Hessian kernel modes 1 and 2; tracer: the two halves of the
// batched product).
static riot_status dual_hvp(riot_ctx *ctx, const double *W, double *Y, int m)
{
    const int n = ctx->n, p = ctx->p;
    cudaStream_t s = ctx->s;
    CU(cudaMemcpyAsync(ctx->psF, W, sizeof(double) * (size_t)p * m, cudaMemcpyDeviceToDevice, s));
    CU(scale_rows(p, m, p, ctx->psS, ctx->psF, 1, s));
    if (ctx->model == RIOT_MODEL_ADVDIFF) {
        CU(adv_ad(ctx->a, ctx->psF, m, ctx->U, n, s));
        CU(adv_tl(ctx->a, ctx->U, n, m, ctx->psR, s));
    } else {
        CU(l96_hvp_launch_f64(ctx->m, ctx->coef64, nullptr, ctx->U, n, m, 0, ctx->psF, 1, s));
        CU(l96_hvp_launch_f64(ctx->m, ctx->coef64, ctx->U, nullptr, n, m, 0, ctx->psR, 2, s));
    }
    CU(cudaMemcpyAsync(Y, ctx->psR, sizeof(double) * (size_t)p * m, cudaMemcpyDeviceToDevice, s));
    CU(scale_rows(p, m, p, ctx->psSig, Y, 1, s));
    return RIOT_OK;
}

riot_status riot_psas(riot_ctx *ctx, int32_t m, int32_t q, int64_t sketch_stream, const double *Omega_dev,
                      double *lambda_out, double *dv_dev, int32_t *mode_out)
{
    if (!ctx) return RIOT_EINVAL;
    if (!ctx->have_traj) return fail(ctx, RIOT_ESTATE, "riot_psas before riot_outer_begin");
    if (m < 1 || m > ctx->kmax || m > ctx->p)
        return fail(ctx, RIOT_EINVAL, "m = %d outside [1, min(kmax = %d, p = %d)]", m, ctx->kmax, ctx->p);
    if (q < 0 || q > 64) return fail(ctx, RIOT_EINVAL, "q = %d outside [0, 64]", q);
    if (!ctx->pc_m.empty()) return fail(ctx, RIOT_ESTATE, "riot_psas: Algorithm 4 runs without the spectral preconditioner");
    CU(cudaSetDevice(ctx->dev));
    TRY(psas_alloc(ctx));
    const int n = ctx->n, p = ctx->p;
    cudaStream_t s = ctx->s;
    ctx->have_rsvd = 0;   // the primal Ritz pairs are not kept
    ctx->pc_open = 0;
    // r = S (d - b') with d = y - H(x) (the dual's sign; the context holds H(x) - y) and
    // b' = H (x_b - x) = H L (-v): the tangent linear model of -v (mode 2 gives R^-1 H L (-v))
    CU(cudaMemcpyAsync(ctx->tmp, ctx->v, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    CU(scal(n, -1.0, ctx->tmp, s));
    if (ctx->model == RIOT_MODEL_ADVDIFF) CU(adv_tl_obs(ctx->a, ctx->tmp, ctx->psR, s));
    else CU(l96_hvp_launch_f64(ctx->m, ctx->coef64, ctx->tmp, nullptr, n, 1, 0, ctx->psR, 2, s));
    CU(mul(p, ctx->psS, ctx->d, ctx->psr, s));                 // S (H(x) - y)
    CU(mul(p, ctx->psSig, ctx->psR, ctx->psw, s));             // S b' = sigma_o (R^-1 b')
    CU(axpby(p, -1.0, ctx->psw, -1.0, ctx->psr, s));           // r = -S (H(x) - y) - S b'
    // sketch, products, power iterations, basis
    CU(cudaMemsetAsync(ctx->info, 0, sizeof(int) * 32, s));
    if (Omega_dev)
        CU(cudaMemcpyAsync(ctx->psW, Omega_dev, sizeof(double) * (size_t)p * m, cudaMemcpyDeviceToDevice, s));
    else
        CU(normal_launch(ctx->seed, (uint32_t)sketch_stream, p, m, p, 1, ctx->psW, s));
    TRY(dual_hvp(ctx, ctx->psW, ctx->psY, m));
    for (int it = 0; it < q; ++it) {
        CU(cudaMemcpyAsync(ctx->psW, ctx->psY, sizeof(double) * (size_t)p * m, cudaMemcpyDeviceToDevice, s));
        TRY(cholqr64(ctx, ctx->psW, m, 3, 0, p));
        TRY(dual_hvp(ctx, ctx->psW, ctx->psY, m));
    }
    CU(cudaMemcpyAsync(ctx->psQ, ctx->psY, sizeof(double) * (size_t)p * m, cudaMemcpyDeviceToDevice, s));
    TRY(cholqr64(ctx, ctx->psQ, m, 3, 5, p));
    TRY(check_cholesky(ctx, 0, 10, "riot_psas"));
    // K: Q^T A Q (exact_rr) or K (Q^T W) = Q^T Y through K (M M^T) = N M^T, symmetrised
    if (ctx->exact_rr) {
        TRY(dual_hvp(ctx, ctx->psQ, ctx->psY, m));
        CU(gemm('T', 'N', m, m, p, 1.0, ctx->psQ, 'd', p, ctx->psY, 'd', p, 0.0, ctx->Km, 'd', m, s));
    } else {
        CU(gemm('T', 'N', m, m, p, 1.0, ctx->psQ, 'd', p, ctx->psW, 'd', p, 0.0, ctx->Mm, 'd', m, s));
        CU(gemm('T', 'N', m, m, p, 1.0, ctx->psQ, 'd', p, ctx->psY, 'd', p, 0.0, ctx->Nm, 'd', m, s));
        for (int attempt = 0; attempt < 2; ++attempt) {
            CU(syrk_lower(m, m, ctx->Mm, m, ctx->G, m, s));
            CU(gemm('N', 'T', m, m, m, 1.0, ctx->Nm, 'd', m, ctx->Mm, 'd', m, 0.0, ctx->Km, 'd', m, s));
            CU(cudaMemsetAsync(ctx->info + 10, 0, sizeof(int), s));
            CU(cholesky(ctx->G, m, m, attempt ? 8.0 * m * ldexp(1.0, -53) : 0.0, ctx->info + 10, ctx->gws, s,
                        ctx->chol_whole_gpu));
            CU(trsm_right_lt(ctx->Km, m, m, m, ctx->G, m, s, ctx->gws));
            CU(trsm_right_l(ctx->Km, m, m, m, ctx->G, m, s, ctx->gws));
            int i10 = 0;
            CU(cudaMemcpyAsync(&i10, ctx->info + 10, sizeof(int), cudaMemcpyDeviceToHost, s));
            CU(cudaStreamSynchronize(s));
            if (i10 == 0) break;
            if (attempt) return fail(ctx, RIOT_ENOTSPD, "riot_psas: the solve for K failed (Q^T W singular)");
        }
    }
    CU(symmetrize(ctx->Km, m, m, s));
    TRY(small_eig(ctx, m, "riot_psas"));
    CU(gemm('N', 'N', p, m, m, 1.0, ctx->psQ, 'd', p, ctx->Z, 'd', m, 0.0, ctx->psU, 'd', p, s));
    CU(fix_col_signs(ctx->psU, p, m, p, s));
    // adaptive weights: LRA w = U diag(1/(1+lambda)) U^T r, LRU w = r - U diag(lambda/(1+lambda)) U^T r
    CU(gemm('T', 'N', m, 1, p, 1.0, ctx->psU, 'd', p, ctx->psr, 'd', p, 0.0, ctx->psc, 'd', m, s));
    CU(cov_coef(ctx->lam, m, ctx->cvec, ctx->info + 14, s));
    CU(mul(m, ctx->cvec, ctx->psc, ctx->psc, s));
    int mode = 0;
    CU(cudaMemcpyAsync(&mode, ctx->info + 14, sizeof(int), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    if (mode == 0) {
        CU(gemm('N', 'N', p, 1, m, 1.0, ctx->psU, 'd', p, ctx->psc, 'd', m, 0.0, ctx->psw, 'd', p, s));
    } else {
        CU(cudaMemcpyAsync(ctx->psw, ctx->psr, sizeof(double) * p, cudaMemcpyDeviceToDevice, s));
        CU(gemm('N', 'N', p, 1, m, -1.0, ctx->psU, 'd', p, ctx->psc, 'd', m, 1.0, ctx->psw, 'd', p, s));
    }
    CU(mul(p, ctx->psS, ctx->psw, ctx->psF, s));               // dw = S w
    // x = x_b + B H^T dw = x_b + L v with v = L^T H^T dw (one adjoint run); dv = v_new - v
    if (ctx->model == RIOT_MODEL_ADVDIFF) CU(adv_ad_obs(ctx->a, ctx->psF, ctx->tmp, s));
    else CU(l96_hvp_launch_f64(ctx->m, ctx->coef64, nullptr, ctx->tmp, n, 1, 0, ctx->psF, 1, s));
    CU(cudaMemcpyAsync(ctx->dv, ctx->tmp, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    CU(axpby(n, -1.0, ctx->v, 1.0, ctx->dv, s));
    CU(cudaMemcpyAsync(ctx->v, ctx->tmp, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    CU(bsqrt(ctx, ctx->dv, ctx->tmp, 0, 1));
    CU(axpby(n, 1.0, ctx->tmp, 1.0, ctx->x, s));
    if (dv_dev) CU(cudaMemcpyAsync(dv_dev, ctx->dv, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    if (lambda_out) CU(cudaMemcpyAsync(lambda_out, ctx->lam, sizeof(double) * m, cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    if (mode_out) *mode_out = mode;
    return RIOT_OK;
}

riot_status riot_precond_enable(riot_ctx *ctx, int32_t max_cols, int32_t rotation)
{
    if (!ctx) return RIOT_EINVAL;
    if (max_cols < 0 || max_cols > ctx->n) return fail(ctx, RIOT_EINVAL, "max_cols = %d outside [0, n = %d]", max_cols, ctx->n);
    CU(cudaSetDevice(ctx->dev));
    CU(cudaStreamSynchronize(ctx->s));   // queued work may still read the old factors
    // dropping factors leaves a gradient formed with them stale (riot_outer_begin again);
    // the state of the current inner loop (rsvd / increment done) is kept
    if (!ctx->pc_m.empty()) ctx->pc_dirty = 1;
    pc_free(ctx);
    if (max_cols == 0) return RIOT_OK;
    const size_t n = (size_t)ctx->n, cap = (size_t)max_cols, kk = (size_t)ctx->kmax * ctx->kmax;
    const bool mixed = (ctx->prec == RIOT_PREC_MIXED);
    riot_status st;
    if ((st = pc_alloc(ctx, &ctx->pcV, n * cap)) || (st = pc_alloc(ctx, &ctx->pcc, cap)) ||
        (st = pc_alloc(ctx, &ctx->pci, cap)) || (st = pc_alloc(ctx, &ctx->pcT, kk)) ||
        (rotation && (st = pc_alloc(ctx, &ctx->pcB, n * cap))) ||
        (mixed && ((st = pc_alloc(ctx, &ctx->pcV32, n * cap)) || (st = pc_alloc(ctx, &ctx->pcT32, kk)) ||
                   (rotation && (st = pc_alloc(ctx, &ctx->pcB32, n * cap)))))) {
        pc_free(ctx);
        return st;
    }
    ctx->pc_cap = max_cols;
    ctx->pc_rot = rotation ? 1 : 0;
    return RIOT_OK;
}

riot_status riot_precond_push(riot_ctx *ctx, int32_t m)
{
    if (!ctx) return RIOT_EINVAL;
    if (!ctx->pc_cap) return fail(ctx, RIOT_ESTATE, "riot_precond_push before riot_precond_enable");
    if (!ctx->have_rsvd || !ctx->pc_ready)
        return fail(ctx, RIOT_ESTATE, "riot_precond_push takes the pairs of an inner loop after its riot_increment");
    if (m < 1 || m > ctx->k_last) return fail(ctx, RIOT_EINVAL, "m = %d outside [1, k = %d]", m, ctx->k_last);
    CU(cudaSetDevice(ctx->dev));
    std::vector<double> lam(m);
    CU(cudaMemcpyAsync(lam.data(), ctx->lam, sizeof(double) * m, cudaMemcpyDeviceToHost, ctx->s));
    CU(cudaStreamSynchronize(ctx->s));
    TRY(pc_push(ctx, ctx->U, lam.data(), m));
    ctx->pc_ready = 0;
    return RIOT_OK;
}

riot_status riot_precond_push_pairs(riot_ctx *ctx, const double *V_dev, const double *lambda, int32_t m)
{
    if (!ctx) return RIOT_EINVAL;
    if (!ctx->pc_cap) return fail(ctx, RIOT_ESTATE, "riot_precond_push_pairs before riot_precond_enable");
    if (ctx->pc_open) return fail(ctx, RIOT_ESTATE, "riot_precond_push_pairs inside an inner loop (before its riot_increment)");
    if (m < 1 || m > ctx->kmax || !V_dev || !lambda)
        return fail(ctx, RIOT_EINVAL, "m = %d outside [1, kmax = %d] or null pairs", m, ctx->kmax);
    CU(cudaSetDevice(ctx->dev));
    return pc_push(ctx, V_dev, lambda, m);
}

riot_status riot_precond_apply(riot_ctx *ctx, const double *X_dev, double *Y_dev, int32_t ncols, int32_t op)
{
    if (!ctx) return RIOT_EINVAL;
    if (ncols < 0 || (ncols > 0 && (!X_dev || !Y_dev)) || op < PC_P || op > PC_PINV)
        return fail(ctx, RIOT_EINVAL, "riot_precond_apply: bad arguments");
    if (ncols == 0) return RIOT_OK;
    CU(cudaSetDevice(ctx->dev));
    const int n = ctx->n;
    if (X_dev != Y_dev)
        CU(cudaMemcpyAsync(Y_dev, X_dev, sizeof(double) * (size_t)n * ncols, cudaMemcpyDeviceToDevice, ctx->s));
    for (int c0 = 0; c0 < ncols; c0 += ctx->kmax) {
        const int nc = (ncols - c0 < ctx->kmax) ? ncols - c0 : ctx->kmax;
        TRY(pc_apply64(ctx, Y_dev + (size_t)c0 * n, nc, op));
    }
    return RIOT_OK;
}

int32_t riot_precond_count(const riot_ctx *ctx) { return ctx ? (int32_t)ctx->pc_m.size() : -1; }

riot_status riot_tc_gram(int32_t n, int32_t k, const float *Y_dev, int64_t ldy, double *G_dev, int64_t ldg,
                         void *cuda_stream)
{
    if (n < 0 || k < 0) return RIOT_EINVAL;
    if (k == 0) return RIOT_OK;
    if ((n > 0 && !Y_dev) || !G_dev || ldy < (n > 1 ? n : 1) || ldg < k) return RIOT_EINVAL;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    void *ws = nullptr;
    int *err = nullptr;
    if (cudaMalloc(&ws, tc_gram_ws_bytes(k)) != cudaSuccess) return RIOT_ENOMEM;
    if (cudaMalloc(&err, sizeof(int)) != cudaSuccess) {
        cudaFree(ws);
        return RIOT_ENOMEM;
    }
    int herr = 0;
    cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int), s);
    if (e == cudaSuccess) e = tc_gram_f32(n, k, Y_dev, ldy, G_dev, ldg, ws, err, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(ws);
    cudaFree(err);
    if (e != cudaSuccess) return RIOT_ECUDA;
    return herr ? RIOT_ETIMEOUT : RIOT_OK;
}

}  // extern "C"
