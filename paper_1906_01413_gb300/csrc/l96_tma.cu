// FP32 batched Lorenz-96 Hessian-vector kernel with TMA-streamed stage coefficients.
//
// Same mathematics as l96_hvp_kernel (Eq. 4 through one tangent-linear RK4
// integration forward and one adjoint integration backward per sketch
// column, Algorithm 3), arranged for sm_103a:
//  * The per-stage base coefficients (a, b) of a whole state (Np float2) are
//    streamed from global memory into a ring of S shared-memory stage
//    buffers by one thread with cp.async.bulk (the 1-D TMA copy), completion
//    tracked by an mbarrier per buffer.  The copy for stage u + S - 1 is
//    issued as soon as every thread has passed the barrier of stage u, so
//    global-memory latency is hidden behind S - 1 stages of arithmetic and
//    every coefficient is read once per CTA and shared by its P probes.
//  * P probes per CTA (1024 threads for E <= 8) keep their state in
//    registers; halos cross chunk boundaries through shared memory.
//  * Every wait on an mbarrier is bounded; a wait that runs out raises a
//    flag in global memory (reported as RIOT_ETIMEOUT) and the CTA carries
//    on, so the kernel always finishes.
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace riot {

namespace {

__device__ __forceinline__ int swz(int x) { return x + (x >> 3); }
__host__ __device__ __forceinline__ int stage_pad_t(int Np) { return Np + (Np >> 3) + 2; }

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait (about 2^20 polls, well under a second).  After one wait of
// the CTA has run out, later waits return at once: the results are then
// wrong, the flag says so, and the kernel still finishes promptly.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, int *err, volatile int *abort_flag)
{
    if (*abort_flag) return false;
    for (int i = 0; i < (1 << 20); ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if (i > 32) __nanosleep(64);
    }
    *abort_flag = 1;
    atomicExch(err, 1);
    return false;
}

struct TmaArgs {
    ChunkGeom geom;
    int T, P, S, p, hl, hh, ncols, add_identity, mode;
    float dt;
    const float2 *coef;
    const int *optr, *oslot;
    const float *rinv, *band, *sig, *W;
    float *Y, *r;
    long long ld;
    int *err;
};

// Ring of stage buffers fed by thread 0.  Stream position c = 0.. counts the
// stages this launch consumes; stage c of the stream is coefficient block
// blk(c) of the [T][4] array: forward for the tangent-linear pass, backward
// for the adjoint pass.
struct Ring {
    float2 *buf;
    uint32_t bar0;
    int S, Np, total, c0, T;
    const float2 *coef;
    volatile int *abort_flag;
    __device__ int blk(int c) const
    {
        const int u = c0 + c;
        return u < 4 * T ? u : 8 * T - 1 - u;
    }
    __device__ void issue(int c) const
    {
        const int slot = c % S;
        const uint32_t bytes = (uint32_t)Np * 8u;
        const uint32_t bar = bar0 + 8u * slot;
        fence_proxy_async();
        mbar_expect_tx(bar, bytes);
        bulk_g2s(smem_u32(buf + (size_t)slot * Np), coef + (size_t)blk(c) * Np, bytes, bar);
    }
    // Called by every thread right after the stage's barrier: refill, then wait.
    __device__ const float2 *acquire(int c, int *err) const
    {
        if (threadIdx.x == 0 && c + S - 1 < total && !*abort_flag) issue(c + S - 1);
        const int slot = c % S;
        mbar_wait_bounded(bar0 + 8u * slot, (uint32_t)((c / S) & 1), err, abort_flag);
        return buf + (size_t)slot * Np;
    }
    // After an abort: wait (bounded) for the copies this CTA still has in flight.
    __device__ void drain(int next_c, int *err) const
    {
        if (threadIdx.x != 0 || !*abort_flag) return;
        for (int c = next_c; c < total && c < next_c + S - 1; ++c)
            for (int i = 0; i < (1 << 20); ++i)
                if (mbar_try_wait(bar0 + 8u * (c % S), (uint32_t)((c / S) & 1))) break;
    }
};

template <int E>
__device__ __forceinline__ void tl_stage(const float (&s)[E], float (&k)[E], bool full, float *H, int nthr, int tid,
                                         int left, int right, int &hb, const Ring &ring, int c, int tE, int *err)
{
    float *Hb = H + hb * 4 * nthr;
    Hb[tid] = full ? s[E - 2] : s[E - 3];
    Hb[nthr + tid] = full ? s[E - 1] : s[E - 2];
    Hb[2 * nthr + tid] = s[0];
    __syncthreads();
    const float m2 = Hb[left], m1 = Hb[nthr + left], p1 = Hb[2 * nthr + right];
    hb ^= 1;
    const float4 *cf = reinterpret_cast<const float4 *>(ring.acquire(c, err) + tE);
#pragma unroll
    for (int j2 = 0; j2 < E / 2; ++j2) {
        const float4 cc = cf[j2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int j = 2 * j2 + h;
            const float ca = h ? cc.z : cc.x, cb = h ? cc.w : cc.y;
            const float xm2 = (j == 0) ? m2 : (j == 1 ? m1 : s[j >= 2 ? j - 2 : 0]);
            const float xm1 = (j == 0) ? m1 : s[j >= 1 ? j - 1 : 0];
            float xp1;
            if (j == E - 1) xp1 = p1;
            else if (j == E - 2) xp1 = full ? s[E - 1] : p1;
            else xp1 = s[j + 1 < E ? j + 1 : 0];
            k[j] = fmaf(ca, xp1 - xm2, fmaf(cb, xm1, -s[j]));
        }
    }
    if (!full) k[E - 1] = 0.f;
}

template <int E>
__device__ __forceinline__ void ad_stage(const float (&m)[E], float (&out)[E], bool full, float *H, int nthr, int tid,
                                         int left, int right, int &hb, const Ring &ring, int c, int tE, int *err)
{
    // The coefficients are needed before the exchange here (p = a m, q = b m),
    // so the stage waits first; the barrier below still orders the refill.
    const float4 *cf = reinterpret_cast<const float4 *>(ring.acquire(c, err) + tE);
    float pp[E], qq[E];
#pragma unroll
    for (int j2 = 0; j2 < E / 2; ++j2) {
        const float4 cc = cf[j2];
        pp[2 * j2] = cc.x * m[2 * j2];
        qq[2 * j2] = cc.y * m[2 * j2];
        pp[2 * j2 + 1] = cc.z * m[2 * j2 + 1];
        qq[2 * j2 + 1] = cc.w * m[2 * j2 + 1];
    }
    float *Hb = H + hb * 4 * nthr;
    Hb[tid] = full ? pp[E - 1] : pp[E - 2];
    Hb[nthr + tid] = pp[0];
    Hb[2 * nthr + tid] = pp[1];
    Hb[3 * nthr + tid] = qq[0];
    __syncthreads();
    const float pm1 = Hb[left], pR0 = Hb[nthr + right], pR1 = Hb[2 * nthr + right], qR0 = Hb[3 * nthr + right];
    hb ^= 1;
#pragma unroll
    for (int j = 0; j < E; ++j) {
        const float pjm1 = (j == 0) ? pm1 : pp[j >= 1 ? j - 1 : 0];
        float qjp1;
        if (j <= E - 3) qjp1 = qq[j + 1 < E ? j + 1 : 0];
        else if (j == E - 2) qjp1 = full ? qq[E - 1] : qR0;
        else qjp1 = qR0;
        float pjp2;
        if (j <= E - 4) pjp2 = pp[j + 2 < E ? j + 2 : 0];
        else if (j == E - 3) pjp2 = full ? pp[E - 1] : pR0;
        else if (j == E - 2) pjp2 = full ? pR0 : pR1;
        else pjp2 = pR1;
        out[j] = (pjm1 - pjp2) + (qjp1 - m[j]);
    }
    if (!full) out[E - 1] = 0.f;
}

template <int E>
__device__ __forceinline__ void band_apply_t(const float *st, const float *band, int hl, int hh, int n, int s0, int len,
                                             float (&out)[E])
{
#pragma unroll
    for (int j = 0; j < E; ++j) out[j] = 0.f;
    for (int d = -hl; d <= hh; ++d) {
        const float w = band[d + hl];
#pragma unroll
        for (int j = 0; j < E; ++j) {
            int ii = s0 + j + d;
            ii += (ii < 0) ? n : 0;
            ii -= (ii >= n) ? n : 0;
            if (j < len) out[j] = fmaf(w, st[swz(ii)], out[j]);
        }
    }
}

template <int E, int MAXT>
__global__ void __launch_bounds__(MAXT, 1) l96_hvp_tma_kernel(const TmaArgs a)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const ChunkGeom &G = a.geom;
    const int Np = G.Np, n = G.n, Tp = G.Tp, P = a.P, S = a.S;
    const int nthr = blockDim.x;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem_raw);
    float2 *ringbuf = reinterpret_cast<float2 *>(smem_raw + 128);
    float *H = reinterpret_cast<float *>(ringbuf + (size_t)S * Np);
    float *state = H + 8 * nthr;
    const int SP = stage_pad_t(Np);

    const int tid = threadIdx.x;
    const int t = tid / P, pp = tid - t * P;
    const int probe = blockIdx.x * P + pp;
    const bool active = probe < a.ncols;
    const int left = ((t == 0) ? Tp - 1 : t - 1) * P + pp;
    const int right = ((t == Tp - 1) ? 0 : t + 1) * P + pp;
    const int s0 = G.start(t);
    const int len = G.len(t);
    const bool full = (len == E);
    const int tE = t * E;
    float *st = state + pp * SP;
    int hb = 0;
    const float h = a.dt, h2 = 0.5f * a.dt, h6 = a.dt / 6.f, h3 = a.dt / 3.f;
    const size_t rbase = (size_t)(active ? probe : 0) * (size_t)a.p;

    Ring ring;
    ring.buf = ringbuf;
    ring.bar0 = smem_u32(bars);
    ring.S = S;
    ring.Np = Np;
    ring.T = a.T;
    ring.coef = a.coef;
    ring.c0 = (a.mode == 1) ? 4 * a.T : 0;
    ring.total = ((a.mode == 2) ? 4 * a.T : 8 * a.T) - ring.c0;
    __shared__ int abort_flag;
    ring.abort_flag = &abort_flag;
    if (tid == 0) {
        abort_flag = 0;
        for (int i = 0; i < S; ++i) mbar_init(ring.bar0 + 8u * i, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0)
        for (int c = 0; c < S - 1 && c < ring.total; ++c) ring.issue(c);
    int c = 0;   // stream position

    float dx[E];
    if (a.mode != 1) {
        const float *w = a.W + (size_t)(active ? probe : 0) * a.ld;
        for (int i = t; i < n; i += Tp) st[swz(i)] = active ? w[i] : 0.f;
        __syncthreads();
        band_apply_t<E>(st, a.band, a.hl, a.hh, n, s0, len, dx);
#pragma unroll
        for (int j = 0; j < E; ++j) dx[j] = (j < len) ? dx[j] * a.sig[s0 + (j < len ? j : 0)] : 0.f;
        __syncthreads();
        for (int tt = 0;; ++tt) {
            const int o0 = a.optr[tt], o1 = a.optr[tt + 1];
            if (o0 < o1) {
#pragma unroll
                for (int j = 0; j < E; ++j) st[swz(tE + j)] = dx[j];
                __syncthreads();
                if (active)
                    for (int o = o0 + t; o < o1; o += Tp) a.r[rbase + o] = a.rinv[o] * st[swz(a.oslot[o])];
                __syncthreads();
            }
            if (tt == a.T) break;
            float s[E], k[E], acc[E];
#pragma unroll
            for (int j = 0; j < E; ++j) s[j] = dx[j];
            tl_stage<E>(s, k, full, H, nthr, tid, left, right, hb, ring, c++, tE, a.err);
#pragma unroll
            for (int j = 0; j < E; ++j) { acc[j] = k[j]; s[j] = fmaf(h2, k[j], dx[j]); }
            tl_stage<E>(s, k, full, H, nthr, tid, left, right, hb, ring, c++, tE, a.err);
#pragma unroll
            for (int j = 0; j < E; ++j) { acc[j] = fmaf(2.f, k[j], acc[j]); s[j] = fmaf(h2, k[j], dx[j]); }
            tl_stage<E>(s, k, full, H, nthr, tid, left, right, hb, ring, c++, tE, a.err);
#pragma unroll
            for (int j = 0; j < E; ++j) { acc[j] = fmaf(2.f, k[j], acc[j]); s[j] = fmaf(h, k[j], dx[j]); }
            tl_stage<E>(s, k, full, H, nthr, tid, left, right, hb, ring, c++, tE, a.err);
#pragma unroll
            for (int j = 0; j < E; ++j) { acc[j] += k[j]; dx[j] = fmaf(h6, acc[j], dx[j]); }
        }
        if (a.mode == 2) {
            ring.drain(c, a.err);
            return;
        }
        __syncthreads();   // last tangent-linear stage read before the adjoint refills its buffer
    }

    float lam[E];
#pragma unroll
    for (int j = 0; j < E; ++j) lam[j] = 0.f;
    for (int tt = a.T;; --tt) {
        const int o0 = a.optr[tt], o1 = a.optr[tt + 1];
        if (o0 < o1) {
#pragma unroll
            for (int j = 0; j < E; ++j) st[swz(tE + j)] = lam[j];
            __syncthreads();
            if (active)
                for (int o = o0 + t; o < o1; o += Tp) atomicAdd(&st[swz(a.oslot[o])], a.r[rbase + o]);
            __syncthreads();
#pragma unroll
            for (int j = 0; j < E; ++j) lam[j] = (j < len) ? st[swz(tE + j)] : 0.f;
        }
        if (tt == 0) break;
        float lk[E], ls[E], lx[E];
#pragma unroll
        for (int j = 0; j < E; ++j) lk[j] = h6 * lam[j];
        ad_stage<E>(lk, ls, full, H, nthr, tid, left, right, hb, ring, c++, tE, a.err);
#pragma unroll
        for (int j = 0; j < E; ++j) { lx[j] = lam[j] + ls[j]; lk[j] = fmaf(h3, lam[j], h * ls[j]); }
        ad_stage<E>(lk, ls, full, H, nthr, tid, left, right, hb, ring, c++, tE, a.err);
#pragma unroll
        for (int j = 0; j < E; ++j) { lx[j] += ls[j]; lk[j] = fmaf(h3, lam[j], h2 * ls[j]); }
        ad_stage<E>(lk, ls, full, H, nthr, tid, left, right, hb, ring, c++, tE, a.err);
#pragma unroll
        for (int j = 0; j < E; ++j) { lx[j] += ls[j]; lk[j] = fmaf(h6, lam[j], h2 * ls[j]); }
        ad_stage<E>(lk, ls, full, H, nthr, tid, left, right, hb, ring, c++, tE, a.err);
#pragma unroll
        for (int j = 0; j < E; ++j) lam[j] = lx[j] + ls[j];
    }

    ring.drain(c, a.err);
    __syncthreads();
#pragma unroll
    for (int j = 0; j < E; ++j)
        if (j < len) st[swz(s0 + j)] = a.sig[s0 + j] * lam[j];
    __syncthreads();
    float y[E];
    band_apply_t<E>(st, a.band, a.hl, a.hh, n, s0, len, y);
    if (active) {
        float *yo = a.Y + (size_t)probe * a.ld;
        const float *w = a.W ? a.W + (size_t)probe * a.ld : nullptr;
#pragma unroll
        for (int j = 0; j < E; ++j)
            if (j < len) yo[s0 + j] = y[j] + ((a.add_identity && w) ? w[s0 + j] : 0.f);
    }
}

size_t tma_smem_bytes(int Np, int nthr, int P, int S)
{
    return 128 + (size_t)S * Np * 8 + sizeof(float) * (8 * (size_t)nthr + (size_t)P * stage_pad_t(Np));
}

}  // namespace

// Choose P probes per CTA and ring depth S for the shared-memory budget.
static bool tma_plan(const ChunkGeom &g, int ncols, int maxthr, size_t smem_max, int *P_out, int *S_out)
{
    int P = maxthr / g.Tp;
    if (P > 64) P = 64;
    if (P > ncols) P = ncols;
    for (; P >= 1; --P)
        for (int S = 4; S >= 2; --S)
            if (tma_smem_bytes(g.Np, P * g.Tp, P, S) <= smem_max) {
                *P_out = P;
                *S_out = S;
                return true;
            }
    return false;
}

cudaError_t l96_hvp_tma_launch(const L96Dev &m, const float2 *coef, const float *W, float *Y, int64_t ld, int ncols,
                               int add_identity, float *r, int mode, int *err, cudaStream_t s)
{
    if (ncols <= 0) return cudaSuccess;
    int dev = 0, smem_optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const int E = m.geom.E;
    const int maxthr = (E <= 8) ? 1024 : 512;
    int P = 1, S = 2;
    // leave room for the kernel's static shared memory
    if (!tma_plan(m.geom, ncols, maxthr, (size_t)smem_optin - 1024, &P, &S)) return cudaErrorInvalidConfiguration;
    TmaArgs a;
    a.geom = m.geom;
    a.T = m.T;
    a.P = P;
    a.S = S;
    a.p = m.p;
    a.hl = m.band.hl;
    a.hh = m.band.hh;
    a.ncols = ncols;
    a.add_identity = add_identity;
    a.mode = mode;
    a.dt = (float)m.dt;
    a.coef = coef;
    a.optr = m.optr;
    a.oslot = m.oslot;
    a.rinv = m.rinv32;
    a.band = m.band32;
    a.sig = m.sig32;
    a.W = W;
    a.Y = Y;
    a.r = r;
    a.ld = ld;
    a.err = err;
    const int nthr = P * m.geom.Tp;
    const size_t sm = tma_smem_bytes(m.geom.Np, nthr, P, S);
    const int grid = (ncols + P - 1) / P;
    cudaError_t e = cudaSuccess;
    switch (E) {
    case 4:
        e = cudaFuncSetAttribute(l96_hvp_tma_kernel<4, 1024>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e == cudaSuccess) { count_launch(); l96_hvp_tma_kernel<4, 1024><<<grid, nthr, sm, s>>>(a); }
        break;
    case 8:
        e = cudaFuncSetAttribute(l96_hvp_tma_kernel<8, 1024>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e == cudaSuccess) { count_launch(); l96_hvp_tma_kernel<8, 1024><<<grid, nthr, sm, s>>>(a); }
        break;
    case 16:
        e = cudaFuncSetAttribute(l96_hvp_tma_kernel<16, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e == cudaSuccess) { count_launch(); l96_hvp_tma_kernel<16, 512><<<grid, nthr, sm, s>>>(a); }
        break;
    default:
        return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace riot
