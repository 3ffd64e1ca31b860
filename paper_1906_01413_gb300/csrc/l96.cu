// Lorenz-96 kernels of the RIOT inner loop on sm_103a.
//
// Model (Section 3.1): dx_i/dt = (x_{i+1} - x_{i-2}) x_{i-1} - x_i + F on a
// periodic ring, advanced by classical RK4.  The Hessian-vector product of
// Eq. 4, A w = L^T sum_t M_{0->t}^T H_t^T R^-1 H_t M_{0->t} L w, is one
// tangent-linear (TL) integration forward and one adjoint (AD) integration
// backward per sketch column (Algorithm 3, "do in parallel").
//
// Design (one GPU, probe-batched):
//  * A CTA owns P probes (sketch columns) x the whole state.  Thread t of a
//    probe keeps E consecutive variables of that probe in registers for the
//    whole window; the periodic stencil reaches across chunk boundaries
//    through a double-buffered shared-memory halo (3-4 words per thread per
//    RK4 stage, one barrier).
//  * The base trajectory enters as per-stage coefficients (a_i, b_i) =
//    (X_{i-1}, X_{i+1} - X_{i-2}) of every RK4 stage state X, written once per
//    outer iteration by the FP64 nonlinear kernel.  Then the TL tendency is
//    a_i (s_{i+1} - s_{i-2}) + b_i s_{i-1} - s_i and the AD tendency is the
//    gather p_{i-1} - p_{i+2} + q_{i+1} - m_i with p = a m, q = b m: both need
//    only per-element coefficients, loaded as 16-byte vectors from L2.
//  * Observations are gathered (TL) and scattered (AD) through a swizzled
//    shared copy of the state; the TL residuals R^-1 H dx wait in global
//    scratch for the AD pass of the same CTA.
//  * L (banded symmetric circulant times diag(sigma)) is applied in the
//    prologue and L^T in the epilogue of the same kernel, so one launch
//    computes the whole Hessian-vector product.
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace riot {

template <typename real> struct V2;
template <> struct V2<float> { using type = float2; };
template <> struct V2<double> { using type = double2; };

// one pad word every 8 words: conflict-free strided access to the state copy
__device__ __forceinline__ int sw(int x) { return x + (x >> 3); }

__host__ __device__ __forceinline__ int stage_pad(int Np) { return Np + (Np >> 3) + 2; }

bool choose_geom(int n, ChunkGeom *g)
{
    if (n < 16 || n > 8192) return false;
    const int cand[3] = {n > 4096 ? 16 : 8, 8, 4};
    for (int c = 0; c < 3; ++c) {
        int E = cand[c];
        int Tp = (n + E - 1) / E;
        int gg = Tp * E - n;
        if (Tp > 512) continue;
        if (gg <= Tp && E - 1 >= 3) {
            g->n = n; g->E = E; g->Tp = Tp; g->g = gg; g->Np = Tp * E;
            return true;
        }
    }
    return false;
}

// ---------------------------------------------------------------------------
// Halo exchanges.  H holds 2 buffers x 4 arrays x nthr words.
// ---------------------------------------------------------------------------
template <typename real, int E>
__device__ __forceinline__ void xchg_tl(const real (&s)[E], bool full, real *H, int nthr, int tid,
                                        int left, int right, int &hb, real &m2, real &m1, real &p1)
{
    real *Hb = H + hb * 4 * nthr;
    Hb[tid] = full ? s[E - 2] : s[E - 3];
    Hb[nthr + tid] = full ? s[E - 1] : s[E - 2];
    Hb[2 * nthr + tid] = s[0];
    __syncthreads();
    m2 = Hb[left];
    m1 = Hb[nthr + left];
    p1 = Hb[2 * nthr + right];
    hb ^= 1;
}

// TL tendency k = J(X) s with per-element coefficients (a, b) of stage X.
template <typename real, int E>
__device__ __forceinline__ void tl_tend(const real (&s)[E], real (&k)[E], const typename V2<real>::type *cf,
                                        bool full, real *H, int nthr, int tid, int left, int right, int &hb)
{
    real m2, m1, p1;
    xchg_tl<real, E>(s, full, H, nthr, tid, left, right, hb, m2, m1, p1);
#pragma unroll
    for (int j = 0; j < E; ++j) {
        typename V2<real>::type c = cf[j];
        real xm2 = (j == 0) ? m2 : (j == 1 ? m1 : s[j >= 2 ? j - 2 : 0]);
        real xm1 = (j == 0) ? m1 : s[j >= 1 ? j - 1 : 0];
        real xp1;
        if (j == E - 1) xp1 = p1;
        else if (j == E - 2) xp1 = full ? s[E - 1] : p1;
        else xp1 = s[j + 1 < E ? j + 1 : 0];
        k[j] = c.x * (xp1 - xm2) + c.y * xm1 - s[j];
    }
    if (!full) k[E - 1] = real(0);
}

// AD tendency out = J(X)^T m.
template <typename real, int E>
__device__ __forceinline__ void ad_tend(const real (&m)[E], real (&out)[E], const typename V2<real>::type *cf,
                                        bool full, real *H, int nthr, int tid, int left, int right, int &hb)
{
    real pp[E], qq[E];
#pragma unroll
    for (int j = 0; j < E; ++j) {
        typename V2<real>::type c = cf[j];
        pp[j] = c.x * m[j];
        qq[j] = c.y * m[j];
    }
    real *Hb = H + hb * 4 * nthr;
    Hb[tid] = full ? pp[E - 1] : pp[E - 2];
    Hb[nthr + tid] = pp[0];
    Hb[2 * nthr + tid] = pp[1];
    Hb[3 * nthr + tid] = qq[0];
    __syncthreads();
    real pm1 = Hb[left];
    real pR0 = Hb[nthr + right];
    real pR1 = Hb[2 * nthr + right];
    real qR0 = Hb[3 * nthr + right];
    hb ^= 1;
#pragma unroll
    for (int j = 0; j < E; ++j) {
        real pjm1 = (j == 0) ? pm1 : pp[j >= 1 ? j - 1 : 0];
        real qjp1;
        if (j <= E - 3) qjp1 = qq[j + 1 < E ? j + 1 : 0];
        else if (j == E - 2) qjp1 = full ? qq[E - 1] : qR0;
        else qjp1 = qR0;
        real pjp2;
        if (j <= E - 4) pjp2 = pp[j + 2 < E ? j + 2 : 0];
        else if (j == E - 3) pjp2 = full ? pp[E - 1] : pR0;
        else if (j == E - 2) pjp2 = full ? pR0 : pR1;
        else pjp2 = pR1;
        out[j] = pjm1 - pjp2 + qjp1 - m[j];
    }
    if (!full) out[E - 1] = real(0);
}

template <typename real>
struct HvpArgs {
    ChunkGeom geom;
    int T, P, p, hl, hh, ncols, add_identity, mode;
    real dt;
    const typename V2<real>::type *coef;
    const int *optr, *oslot;
    const real *rinv, *band, *sig, *W;
    real *Y, *r;
    long long ld;
};

// Banded circulant apply at own elements: out_j = pre_i * sum_d S_d u_{i+d}
template <typename real, int E>
__device__ __forceinline__ void band_apply(const real *st, const real *band, int hl, int hh, int n, int s0,
                                           int len, real (&out)[E])
{
#pragma unroll
    for (int j = 0; j < E; ++j) out[j] = real(0);
    for (int d = -hl; d <= hh; ++d) {
        real w = band[d + hl];
#pragma unroll
        for (int j = 0; j < E; ++j) {
            int ii = s0 + j + d;
            ii += (ii < 0) ? n : 0;
            ii -= (ii >= n) ? n : 0;
            if (j < len) out[j] += w * st[sw(ii)];
        }
    }
}

template <typename real, int E>
__global__ void __launch_bounds__(512) l96_hvp_kernel(const HvpArgs<real> a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    real *H = reinterpret_cast<real *>(smem_raw);
    const int nthr = blockDim.x;
    const ChunkGeom &G = a.geom;
    const int Np = G.Np, n = G.n, Tp = G.Tp, P = a.P;
    const int SP = stage_pad(Np);
    real *state = H + 8 * nthr;

    const int tid = threadIdx.x;
    const int t = tid / P, pp = tid - (tid / P) * P;
    const int probe = blockIdx.x * P + pp;
    const bool active = probe < a.ncols;
    const int left = ((t == 0) ? Tp - 1 : t - 1) * P + pp;
    const int right = ((t == Tp - 1) ? 0 : t + 1) * P + pp;
    const int s0 = G.start(t);
    const int len = G.len(t);
    const bool full = (len == E);
    real *st = state + pp * SP;
    int hb = 0;
    const real h = a.dt, h2 = real(0.5) * a.dt, h6 = a.dt / real(6), h3 = a.dt / real(3);
    const size_t rbase = (size_t)(active ? probe : 0) * (size_t)a.p;

    real dx[E];
    if (a.mode != 1) {
        // ---- prologue: dx_0 = L w = diag(sigma) S w ----
        const real *w = a.W + (size_t)(active ? probe : 0) * a.ld;
        for (int i = t; i < n; i += Tp) st[sw(i)] = active ? w[i] : real(0);
        __syncthreads();
        band_apply<real, E>(st, a.band, a.hl, a.hh, n, s0, len, dx);
#pragma unroll
        for (int j = 0; j < E; ++j) dx[j] = (j < len) ? dx[j] * a.sig[s0 + (j < len ? j : 0)] : real(0);
        __syncthreads();

        // ---- TL forward ----
        for (int tt = 0;; ++tt) {
            const int o0 = a.optr[tt], o1 = a.optr[tt + 1];
            if (o0 < o1) {
#pragma unroll
                for (int j = 0; j < E; ++j) st[sw(t * E + j)] = dx[j];
                __syncthreads();
                if (active)
                    for (int o = o0 + t; o < o1; o += Tp) a.r[rbase + o] = a.rinv[o] * st[sw(a.oslot[o])];
                __syncthreads();
            }
            if (tt == a.T) break;
            const typename V2<real>::type *cf = a.coef + (size_t)tt * 4 * Np + t * E;
            real s[E], k[E], acc[E];
#pragma unroll
            for (int j = 0; j < E; ++j) s[j] = dx[j];
            tl_tend<real, E>(s, k, cf, full, H, nthr, tid, left, right, hb);
#pragma unroll
            for (int j = 0; j < E; ++j) { acc[j] = k[j]; s[j] = dx[j] + h2 * k[j]; }
            tl_tend<real, E>(s, k, cf + Np, full, H, nthr, tid, left, right, hb);
#pragma unroll
            for (int j = 0; j < E; ++j) { acc[j] += real(2) * k[j]; s[j] = dx[j] + h2 * k[j]; }
            tl_tend<real, E>(s, k, cf + 2 * Np, full, H, nthr, tid, left, right, hb);
#pragma unroll
            for (int j = 0; j < E; ++j) { acc[j] += real(2) * k[j]; s[j] = dx[j] + h * k[j]; }
            tl_tend<real, E>(s, k, cf + 3 * Np, full, H, nthr, tid, left, right, hb);
#pragma unroll
            for (int j = 0; j < E; ++j) { acc[j] += k[j]; dx[j] = dx[j] + h6 * acc[j]; }
        }
        if (a.mode == 2) return;
    }

    // ---- AD backward ----
    real lam[E];
#pragma unroll
    for (int j = 0; j < E; ++j) lam[j] = real(0);
    for (int tt = a.T;; --tt) {
        const int o0 = a.optr[tt], o1 = a.optr[tt + 1];
        if (o0 < o1) {
#pragma unroll
            for (int j = 0; j < E; ++j) st[sw(t * E + j)] = lam[j];
            __syncthreads();
            if (active)
                for (int o = o0 + t; o < o1; o += Tp) atomicAdd(&st[sw(a.oslot[o])], a.r[rbase + o]);
            __syncthreads();
#pragma unroll
            for (int j = 0; j < E; ++j) lam[j] = (j < len) ? st[sw(t * E + j)] : real(0);
        }
        if (tt == 0) break;
        const typename V2<real>::type *cf = a.coef + (size_t)(tt - 1) * 4 * Np + t * E;
        real lk[E], ls[E], lx[E];
#pragma unroll
        for (int j = 0; j < E; ++j) lk[j] = h6 * lam[j];
        ad_tend<real, E>(lk, ls, cf + 3 * Np, full, H, nthr, tid, left, right, hb);
#pragma unroll
        for (int j = 0; j < E; ++j) { lx[j] = lam[j] + ls[j]; lk[j] = h3 * lam[j] + h * ls[j]; }
        ad_tend<real, E>(lk, ls, cf + 2 * Np, full, H, nthr, tid, left, right, hb);
#pragma unroll
        for (int j = 0; j < E; ++j) { lx[j] += ls[j]; lk[j] = h3 * lam[j] + h2 * ls[j]; }
        ad_tend<real, E>(lk, ls, cf + Np, full, H, nthr, tid, left, right, hb);
#pragma unroll
        for (int j = 0; j < E; ++j) { lx[j] += ls[j]; lk[j] = h6 * lam[j] + h2 * ls[j]; }
        ad_tend<real, E>(lk, ls, cf, full, H, nthr, tid, left, right, hb);
#pragma unroll
        for (int j = 0; j < E; ++j) lam[j] = lx[j] + ls[j];
    }

    // ---- epilogue: y = L^T lambda_0 = S diag(sigma) lambda_0 (+ w) ----
    __syncthreads();
#pragma unroll
    for (int j = 0; j < E; ++j)
        if (j < len) st[sw(s0 + j)] = a.sig[s0 + j] * lam[j];
    __syncthreads();
    real y[E];
    band_apply<real, E>(st, a.band, a.hl, a.hh, n, s0, len, y);
    if (active) {
        real *yo = a.Y + (size_t)probe * a.ld;
        const real *w = a.W ? a.W + (size_t)probe * a.ld : nullptr;
#pragma unroll
        for (int j = 0; j < E; ++j)
            if (j < len) yo[s0 + j] = y[j] + ((a.add_identity && w) ? w[s0 + j] : real(0));
    }
}

template <typename real>
static cudaError_t hvp_launch(const L96Dev &m, const typename V2<real>::type *coef, const real *W, real *Y,
                              int64_t ld, int ncols, int add_identity, real *r, int mode,
                              const real *rinv, const real *band, const real *sig, cudaStream_t s)
{
    if (ncols <= 0) return cudaSuccess;
    HvpArgs<real> a;
    a.geom = m.geom;
    a.T = m.T;
    a.p = m.p;
    a.hl = m.band.hl;
    a.hh = m.band.hh;
    a.ncols = ncols;
    a.add_identity = add_identity;
    a.mode = mode;
    a.dt = (real)m.dt;
    a.coef = coef;
    a.optr = m.optr;
    a.oslot = m.oslot;
    a.rinv = rinv;
    a.band = band;
    a.sig = sig;
    a.W = W;
    a.Y = Y;
    a.r = r;
    a.ld = ld;
    const int Tp = m.geom.Tp;
    int P = 512 / Tp;
    if (P < 1) return cudaErrorInvalidConfiguration;
    if (P > ncols) P = ncols;
    if (P > 64) P = 64;
    a.P = P;
    const int nthr = P * Tp;
    const size_t sm = sizeof(real) * (8 * (size_t)nthr + (size_t)P * stage_pad(m.geom.Np));
    const int grid = (ncols + P - 1) / P;
    cudaError_t e = cudaSuccess;
    switch (m.geom.E) {
    case 4:
        e = cudaFuncSetAttribute(l96_hvp_kernel<real, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e == cudaSuccess) { count_launch(); l96_hvp_kernel<real, 4><<<grid, nthr, sm, s>>>(a); }
        break;
    case 8:
        e = cudaFuncSetAttribute(l96_hvp_kernel<real, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e == cudaSuccess) { count_launch(); l96_hvp_kernel<real, 8><<<grid, nthr, sm, s>>>(a); }
        break;
    case 16:
        e = cudaFuncSetAttribute(l96_hvp_kernel<real, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e == cudaSuccess) { count_launch(); l96_hvp_kernel<real, 16><<<grid, nthr, sm, s>>>(a); }
        break;
    default:
        return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t l96_hvp_launch_f64(const L96Dev &m, const double2 *coef, const double *W, double *Y, int64_t ld,
                               int ncols, int add_identity, double *r, int mode, cudaStream_t s)
{
    return hvp_launch<double>(m, coef, W, Y, ld, ncols, add_identity, r, mode, m.rinv64, m.band64, m.sig64, s);
}

// ---------------------------------------------------------------------------
// Nonlinear FP64 trajectory + stage coefficients + innovation (one CTA).
// ---------------------------------------------------------------------------
struct NlArgs {
    ChunkGeom geom;
    int T, p;
    double dt, F;
    const int *optr, *oslot;
    const double *y, *rinv, *x0;
    double *traj, *d, *jo, *xT;
    float2 *coef32;
    double2 *coef64;
};

template <int E>
__global__ void __launch_bounds__(512) l96_nl_kernel(const NlArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double *H = reinterpret_cast<double *>(smem_raw);
    const int nthr = blockDim.x;
    double *st = H + 8 * nthr;
    const ChunkGeom &G = a.geom;
    const int Np = G.Np, n = G.n, Tp = G.Tp;
    const int t = threadIdx.x, tid = threadIdx.x;
    const int left = (t == 0) ? Tp - 1 : t - 1, right = (t == Tp - 1) ? 0 : t + 1;
    const int s0 = G.start(t), len = G.len(t);
    const bool full = (len == E);
    int hb = 0;
    const double h = a.dt, h2 = 0.5 * a.dt, h6 = a.dt / 6.0, F = a.F;
    double jsum = 0.0;

    double x[E];
#pragma unroll
    for (int j = 0; j < E; ++j) x[j] = (j < len) ? a.x0[s0 + (j < len ? j : 0)] : 0.0;

    for (int tt = 0;; ++tt) {
        if (a.traj) {
#pragma unroll
            for (int j = 0; j < E; ++j)
                if (j < len) a.traj[(size_t)tt * n + s0 + j] = x[j];
        }
        const int o0 = a.p ? a.optr[tt] : 0, o1 = a.p ? a.optr[tt + 1] : 0;
        if (o0 < o1) {
#pragma unroll
            for (int j = 0; j < E; ++j) st[sw(t * E + j)] = x[j];
            __syncthreads();
            for (int o = o0 + t; o < o1; o += Tp) {
                double dd = st[sw(a.oslot[o])] - a.y[o];
                if (a.d) a.d[o] = dd;
                jsum += 0.5 * dd * dd * a.rinv[o];
            }
            __syncthreads();
        }
        if (tt == a.T) break;
        double X[E], acc[E];
#pragma unroll
        for (int j = 0; j < E; ++j) X[j] = x[j];
#pragma unroll 1
        for (int stage = 0; stage < 4; ++stage) {
            double m2, m1, p1;
            xchg_tl<double, E>(X, full, H, nthr, tid, left, right, hb, m2, m1, p1);
            double f[E];
            const size_t cbase = ((size_t)tt * 4 + stage) * Np + (size_t)t * E;
#pragma unroll
            for (int j = 0; j < E; ++j) {
                double xm2 = (j == 0) ? m2 : (j == 1 ? m1 : X[j >= 2 ? j - 2 : 0]);
                double xm1 = (j == 0) ? m1 : X[j >= 1 ? j - 1 : 0];
                double xp1;
                if (j == E - 1) xp1 = p1;
                else if (j == E - 2) xp1 = full ? X[E - 1] : p1;
                else xp1 = X[j + 1 < E ? j + 1 : 0];
                double ca = xm1, cb = xp1 - xm2;
                f[j] = cb * ca - X[j] + F;
                if (j == E - 1 && !full) { ca = 0.0; cb = 0.0; f[j] = 0.0; }
                // FP32 copy interleaved by element pair across threads: float4 index
                // (j / 2) * Tp + t within the stage, so that the FP32 kernel's
                // shared-memory reads of one pair are contiguous across threads
                if (a.coef32)
                    a.coef32[((size_t)tt * 4 + stage) * Np + (size_t)(j >> 1) * 2 * Tp + 2 * t + (j & 1)] =
                        make_float2((float)ca, (float)cb);
                if (a.coef64) a.coef64[cbase + j] = make_double2(ca, cb);
            }
            const double c = (stage == 2) ? h : h2;
            const double wgt = (stage == 0 || stage == 3) ? 1.0 : 2.0;
#pragma unroll
            for (int j = 0; j < E; ++j) {
                acc[j] = (stage == 0) ? f[j] : acc[j] + wgt * f[j];
                X[j] = x[j] + c * f[j];
            }
        }
#pragma unroll
        for (int j = 0; j < E; ++j) x[j] = full || j < E - 1 ? x[j] + h6 * acc[j] : 0.0;
    }
    if (a.xT) {
#pragma unroll
        for (int j = 0; j < E; ++j)
            if (j < len) a.xT[s0 + j] = x[j];
    }
    if (a.jo) {
        // block reduction of jsum
        __syncthreads();
        for (int off = 16; off > 0; off >>= 1) jsum += __shfl_down_sync(0xffffffffu, jsum, off);
        if ((tid & 31) == 0) st[tid >> 5] = jsum;
        __syncthreads();
        if (tid == 0) {
            double s = 0.0;
            for (int w = 0; w < (nthr + 31) / 32; ++w) s += st[w];
            atomicAdd(a.jo, s);
        }
    }
}

cudaError_t l96_nl_launch(const L96Dev &m, const double *x0, double *traj, float2 *coef32, double2 *coef64,
                          double *d, double *jo, double *xT, cudaStream_t s)
{
    NlArgs a;
    a.geom = m.geom;
    a.T = m.T;
    a.p = m.p;
    a.dt = m.dt;
    a.F = m.F;
    a.optr = m.optr;
    a.oslot = m.oslot;
    a.y = m.y;
    a.rinv = m.rinv64;
    a.x0 = x0;
    a.traj = traj;
    a.d = d;
    a.jo = jo;
    a.xT = xT;
    a.coef32 = coef32;
    a.coef64 = coef64;
    const int nthr = m.geom.Tp;
    if (nthr > 512) return cudaErrorInvalidConfiguration;
    const size_t sm = sizeof(double) * (8 * (size_t)nthr + stage_pad(m.geom.Np));
    cudaError_t e = cudaSuccess;
    switch (m.geom.E) {
    case 4:
        e = cudaFuncSetAttribute(l96_nl_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e == cudaSuccess) { count_launch(); l96_nl_kernel<4><<<1, nthr, sm, s>>>(a); }
        break;
    case 8:
        e = cudaFuncSetAttribute(l96_nl_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e == cudaSuccess) { count_launch(); l96_nl_kernel<8><<<1, nthr, sm, s>>>(a); }
        break;
    case 16:
        e = cudaFuncSetAttribute(l96_nl_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e == cudaSuccess) { count_launch(); l96_nl_kernel<16><<<1, nthr, sm, s>>>(a); }
        break;
    default:
        return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Standalone L / L^T application in FP64 (outer-loop update, covariance).
// ---------------------------------------------------------------------------
__global__ void bsqrt_kernel(int n, int ncols, int hl, int hh, const double *band, const double *sig,
                             const double *in, double *out, int transpose)
{
    const int64_t total = (int64_t)n * ncols;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int col = (int)(idx / n), i = (int)(idx - (int64_t)col * n);
        const double *x = in + (size_t)col * n;
        double acc = 0.0;
        for (int d = -hl; d <= hh; ++d) {
            int ii = i + d;
            ii += (ii < 0) ? n : 0;
            ii -= (ii >= n) ? n : 0;
            acc += band[d + hl] * (transpose ? sig[ii] * x[ii] : x[ii]);
        }
        out[(size_t)col * n + i] = transpose ? acc : sig[i] * acc;
    }
}

cudaError_t bsqrt_launch(const L96Dev &m, const double *in, double *out, int transpose, int ncols, cudaStream_t s)
{
    if (ncols <= 0) return cudaSuccess;
    const int64_t total = (int64_t)m.geom.n * ncols;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    count_launch();
    bsqrt_kernel<<<blocks, 256, 0, s>>>(m.geom.n, ncols, m.band.hl, m.band.hh, m.band64, m.sig64, in, out,
                                        transpose);
    return cudaGetLastError();
}

}  // namespace riot
