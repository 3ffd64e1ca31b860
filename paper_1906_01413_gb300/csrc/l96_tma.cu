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

#include <algorithm>
#include <vector>

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

__device__ __forceinline__ void mbar_inval(uint32_t bar)
{
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(bar) : "memory");
}

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

// Bounded wait of at most `polls` polls (default kWaitPolls, about 2^20 polls,
// well under a second).  After one wait of the CTA has run out, later waits
// return at once: the results are then wrong, the flag says so (value 1),
// and the kernel still finishes promptly.
constexpr int kWaitPolls = 1 << 20;

__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, int *err, volatile int *abort_flag,
                                                  int polls)
{
    if (*abort_flag) return false;
    for (int i = 0; i < polls; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if (i > 32) __nanosleep(64);
    }
    *abort_flag = 1;
    atomicMax(err, 1);
    return false;
}

struct TmaArgs {
    ChunkGeom geom;
    int T, P, S, p, hl, hh, ncols, add_identity, mode;
    int wait_polls;   // poll bound of each wait on a stage copy (kWaitPolls unless a test lowers it)
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
// for the adjoint pass.  Thread 0 keeps `issued` (copies started) and
// `landed` (stages whose copy it has seen complete) so that after an abort it
// can still wait for every copy it started before the CTA exits.
struct Ring {
    float2 *buf;
    uint32_t bar0;
    int S, Np, total, c0, T, polls;
    int issued, landed;
    const float2 *coef;
    volatile int *abort_flag;
    __device__ int blk(int c) const
    {
        const int u = c0 + c;
        return u < 4 * T ? u : 8 * T - 1 - u;
    }
    __device__ void issue(int c)
    {
        const int slot = c % S;
        const uint32_t bytes = (uint32_t)Np * 8u;
        const uint32_t bar = bar0 + 8u * slot;
        fence_proxy_async();
        mbar_expect_tx(bar, bytes);
        bulk_g2s(smem_u32(buf + (size_t)slot * Np), coef + (size_t)blk(c) * Np, bytes, bar);
        issued = c + 1;
    }
    // Thread 0 only, before the stage's barrier: wait until stage c has landed.
    // The barrier then makes the buffer visible to every thread.
    __device__ void wait_ready(int c, int *err)
    {
        if (threadIdx.x == 0 && mbar_wait_bounded(bar0 + 8u * (c % S), (uint32_t)((c / S) & 1), err, abort_flag, polls))
            landed = c + 1;
    }
    // Thread 0 only, after the stage's barrier (every thread is done with the
    // buffer of stage c - 1): refill that buffer with stage c + S - 1.
    __device__ void refill(int c)
    {
        if (threadIdx.x == 0 && c + S - 1 < total && !*abort_flag) issue(c + S - 1);
    }
    __device__ const float4 *slot4(int slot) const { return reinterpret_cast<const float4 *>(buf + (size_t)slot * Np); }
    // After an abort: wait, with the full bound whatever the test limit, for every
    // copy this CTA started and has not seen land.  Each such stage sits in its own
    // buffer (a buffer is refilled only after its previous stage landed), so its
    // phase parity identifies it.  A copy still in flight after that raises the
    // flag to 2: it may land in shared memory the CTA no longer owns.
    __device__ void drain(int *err)
    {
        if (threadIdx.x != 0 || !*abort_flag) return;
        for (int c = landed; c < issued; ++c) {
            bool done = false;
            for (int i = 0; i < kWaitPolls && !done; ++i) {
                done = mbar_try_wait(bar0 + 8u * (c % S), (uint32_t)((c / S) & 1));
                if (!done && i > 32) __nanosleep(64);
            }
            if (!done) atomicMax(err, 2);
        }
    }
};

// Tangent-linear tendency k = J(X) s of one RK4 stage for the PR probes a
// thread holds; coefficients of the stage come from ring buffer `slot`
// (float4 pairs interleaved by thread) and are shared by the PR probes.
template <int E, int PR>
__device__ __forceinline__ void tl_stage(const float (&s)[PR][E], float (&k)[PR][E], bool full, float *H, int nthr,
                                         int tid, int left, int right, int &hb, Ring &ring, int c, int slot, int t,
                                         int Tp, int *err)
{
    float *Hb = H + hb * 3 * PR * nthr;
#pragma unroll
    for (int r = 0; r < PR; ++r) {
        Hb[(0 * PR + r) * nthr + tid] = full ? s[r][E - 2] : s[r][E - 3];
        Hb[(1 * PR + r) * nthr + tid] = full ? s[r][E - 1] : s[r][E - 2];
        Hb[(2 * PR + r) * nthr + tid] = s[r][0];
    }
    ring.wait_ready(c, err);
    __syncthreads();
    ring.refill(c);
    float m2[PR], m1[PR], p1[PR];
#pragma unroll
    for (int r = 0; r < PR; ++r) {
        m2[r] = Hb[(0 * PR + r) * nthr + left];
        m1[r] = Hb[(1 * PR + r) * nthr + left];
        p1[r] = Hb[(2 * PR + r) * nthr + right];
    }
    hb ^= 1;
    const float4 *cf = ring.slot4(slot) + t;
#pragma unroll
    for (int j2 = 0; j2 < E / 2; ++j2) {
        const float4 cc = cf[j2 * Tp];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int j = 2 * j2 + h;
            const float ca = h ? cc.z : cc.x, cb = h ? cc.w : cc.y;
#pragma unroll
            for (int r = 0; r < PR; ++r) {
                const float xm2 = (j == 0) ? m2[r] : (j == 1 ? m1[r] : s[r][j >= 2 ? j - 2 : 0]);
                const float xm1 = (j == 0) ? m1[r] : s[r][j >= 1 ? j - 1 : 0];
                float xp1;
                if (j == E - 1) xp1 = p1[r];
                else if (j == E - 2) xp1 = full ? s[r][E - 1] : p1[r];
                else xp1 = s[r][j + 1 < E ? j + 1 : 0];
                k[r][j] = fmaf(ca, xp1 - xm2, fmaf(cb, xm1, -s[r][j]));
            }
        }
    }
    if (!full)
#pragma unroll
        for (int r = 0; r < PR; ++r) k[r][E - 1] = 0.f;
}

// Adjoint tendency out = J(X)^T m.  The boundary values of m are exchanged
// and the neighbours' coefficients read from the shared ring, so every
// coefficient read follows the stage's barrier.
template <int E, int PR>
__device__ __forceinline__ void ad_stage(const float (&m)[PR][E], float (&out)[PR][E], bool full, float *H, int nthr,
                                         int tid, int left, int right, int &hb, Ring &ring, int c, int slot, int t,
                                         int Tp, int offL, int oddL, int tr, int *err)
{
    float *Hb = H + hb * 3 * PR * nthr;
#pragma unroll
    for (int r = 0; r < PR; ++r) {
        Hb[(0 * PR + r) * nthr + tid] = full ? m[r][E - 1] : m[r][E - 2];
        Hb[(1 * PR + r) * nthr + tid] = m[r][0];
        Hb[(2 * PR + r) * nthr + tid] = m[r][1];
    }
    ring.wait_ready(c, err);
    __syncthreads();
    ring.refill(c);
    float mL[PR], mR0[PR], mR1[PR];
#pragma unroll
    for (int r = 0; r < PR; ++r) {
        mL[r] = Hb[(0 * PR + r) * nthr + left];
        mR0[r] = Hb[(1 * PR + r) * nthr + right];
        mR1[r] = Hb[(2 * PR + r) * nthr + right];
    }
    hb ^= 1;
    const float4 *s4 = ring.slot4(slot);
    const float4 cl = s4[offL], cr = s4[tr];
    const float aL = oddL ? cl.z : cl.x;
    float ca[E], cb[E];
#pragma unroll
    for (int j2 = 0; j2 < E / 2; ++j2) {
        const float4 cc = s4[j2 * Tp + t];
        ca[2 * j2] = cc.x;
        cb[2 * j2] = cc.y;
        ca[2 * j2 + 1] = cc.z;
        cb[2 * j2 + 1] = cc.w;
    }
    // (J^T m)_j = a_{j-1} m_{j-1} - a_{j+2} m_{j+2} + b_{j+1} m_{j+1} - m_j, three FMAs
#pragma unroll
    for (int r = 0; r < PR; ++r) {
#pragma unroll
        for (int j = 0; j < E; ++j) {
            const float mm1 = (j == 0) ? mL[r] : m[r][j >= 1 ? j - 1 : 0];
            const float am1 = (j == 0) ? aL : ca[j >= 1 ? j - 1 : 0];
            float mp1, bp1;
            if (j <= E - 2 && (full || j <= E - 3)) {
                mp1 = m[r][j + 1 < E ? j + 1 : 0];
                bp1 = cb[j + 1 < E ? j + 1 : 0];
            } else {
                mp1 = mR0[r];
                bp1 = cr.y;
            }
            float mp2, ap2;
            if (j <= E - 3 && (full || j <= E - 4)) {
                mp2 = m[r][j + 2 < E ? j + 2 : 0];
                ap2 = ca[j + 2 < E ? j + 2 : 0];
            } else if (full ? (j == E - 2) : (j == E - 3)) {
                mp2 = mR0[r];
                ap2 = cr.x;
            } else {
                mp2 = mR1[r];
                ap2 = cr.z;
            }
            out[r][j] = fmaf(am1, mm1, fmaf(-ap2, mp2, fmaf(bp1, mp1, -m[r][j])));
        }
        if (!full) out[r][E - 1] = 0.f;
    }
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

// A CTA holds P thread groups of Tp threads; group g owns probes
// blk * P * PR + g * PR + r, r < PR, and thread t of a group keeps chunk t of
// each of them in registers.  Threads from P * Tp up to blockDim.x (a
// persistent batch kernel runs windows of several sizes in one block shape)
// are idle: they follow the barriers and touch only their own halo slots.
template <int E, int PR, bool RAGGED = true>
__device__ __forceinline__ void hvp_tma_body(const TmaArgs &a, int blk, unsigned char *smem_raw, int *abort_flag)
{
    const ChunkGeom &G = a.geom;
    const int Np = G.Np, n = G.n, Tp = G.Tp, P = a.P, S = a.S;
    const int nthr = blockDim.x;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem_raw);
    float2 *ringbuf = reinterpret_cast<float2 *>(smem_raw + 128);
    float *H = reinterpret_cast<float *>(ringbuf + (size_t)S * Np);
    float *state = H + 2 * 3 * PR * nthr;
    const int SP = stage_pad_t(Np);

    const int tid = threadIdx.x;
    const bool live = tid < P * Tp;
    const int t = live ? tid / P : 0, g = live ? tid - (tid / P) * P : 0;
    const int probe0 = (blk * P + g) * PR;
    const int left = ((t == 0) ? Tp - 1 : t - 1) * P + g;
    const int right = ((t == Tp - 1) ? 0 : t + 1) * P + g;
    const int s0 = G.start(t);
    const int len = G.len(t);
    const bool full = !RAGGED || (len == E);   // RAGGED = false: every chunk has E variables
    const int tE = t * E;
    const int tl = (t == 0) ? Tp - 1 : t - 1, tr = (t == Tp - 1) ? 0 : t + 1;
    const int lenL = G.len(tl);
    const int offL = ((lenL - 1) >> 1) * Tp + tl, oddL = (lenL - 1) & 1;
    int hb = 0;
    const float h = a.dt, h2 = 0.5f * a.dt, h6 = a.dt / 6.f, h3 = a.dt / 3.f;

    Ring ring;
    ring.buf = ringbuf;
    ring.bar0 = smem_u32(bars);
    ring.S = S;
    ring.Np = Np;
    ring.T = a.T;
    ring.coef = a.coef;
    ring.c0 = (a.mode == 1) ? 4 * a.T : 0;
    ring.total = ((a.mode == 2) ? 4 * a.T : 8 * a.T) - ring.c0;
    ring.polls = a.wait_polls;
    ring.issued = 0;
    ring.landed = 0;
    ring.abort_flag = abort_flag;
    if (tid == 0) {
        for (int i = 0; i < S; ++i) mbar_init(ring.bar0 + 8u * i, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0)
        for (int c = 0; c < S - 1 && c < ring.total; ++c) ring.issue(c);
    int c = 0;      // stream position
    int slot = 0;   // ring buffer of stream position c (c mod S)

    float dx[PR][E];
    if (a.mode != 1) {
#pragma unroll
        for (int r = 0; r < PR; ++r) {
            const int probe = probe0 + r;
            const bool active = probe < a.ncols;
            float *st = state + (g * PR + r) * SP;
            const float *w = a.W + (size_t)(active ? probe : 0) * a.ld;
            if (live)
                for (int i = t; i < n; i += Tp) st[swz(i)] = active ? w[i] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < PR; ++r) {
            float tmp[E];
            band_apply_t<E>(state + (g * PR + r) * SP, a.band, a.hl, a.hh, n, s0, len, tmp);
#pragma unroll
            for (int j = 0; j < E; ++j) dx[r][j] = (j < len) ? tmp[j] * a.sig[s0 + (j < len ? j : 0)] : 0.f;
        }
        __syncthreads();
        for (int tt = 0;; ++tt) {
            const int o0 = a.optr[tt], o1 = a.optr[tt + 1];
            if (o0 < o1) {
                if (live)
#pragma unroll
                    for (int r = 0; r < PR; ++r) {
                        float *st = state + (g * PR + r) * SP;
#pragma unroll
                        for (int j = 0; j < E; ++j) st[swz(tE + j)] = dx[r][j];
                    }
                __syncthreads();
#pragma unroll
                for (int r = 0; r < PR; ++r) {
                    const int probe = probe0 + r;
                    if (live && probe < a.ncols) {
                        const float *st = state + (g * PR + r) * SP;
                        float *rr = a.r + (size_t)probe * (size_t)a.p;
                        for (int o = o0 + t; o < o1; o += Tp) rr[o] = a.rinv[o] * st[swz(a.oslot[o])];
                    }
                }
                __syncthreads();
            }
            if (tt == a.T) break;
            float s[PR][E], k[PR][E], acc[PR][E];
#pragma unroll
            for (int r = 0; r < PR; ++r)
#pragma unroll
                for (int j = 0; j < E; ++j) s[r][j] = dx[r][j];
            tl_stage<E, PR>(s, k, full, H, nthr, tid, left, right, hb, ring, c++, slot, t, Tp, a.err);
            slot = (slot + 1 == S) ? 0 : slot + 1;
#pragma unroll
            for (int r = 0; r < PR; ++r)
#pragma unroll
                for (int j = 0; j < E; ++j) { acc[r][j] = k[r][j]; s[r][j] = fmaf(h2, k[r][j], dx[r][j]); }
            tl_stage<E, PR>(s, k, full, H, nthr, tid, left, right, hb, ring, c++, slot, t, Tp, a.err);
            slot = (slot + 1 == S) ? 0 : slot + 1;
#pragma unroll
            for (int r = 0; r < PR; ++r)
#pragma unroll
                for (int j = 0; j < E; ++j) { acc[r][j] = fmaf(2.f, k[r][j], acc[r][j]); s[r][j] = fmaf(h2, k[r][j], dx[r][j]); }
            tl_stage<E, PR>(s, k, full, H, nthr, tid, left, right, hb, ring, c++, slot, t, Tp, a.err);
            slot = (slot + 1 == S) ? 0 : slot + 1;
#pragma unroll
            for (int r = 0; r < PR; ++r)
#pragma unroll
                for (int j = 0; j < E; ++j) { acc[r][j] = fmaf(2.f, k[r][j], acc[r][j]); s[r][j] = fmaf(h, k[r][j], dx[r][j]); }
            tl_stage<E, PR>(s, k, full, H, nthr, tid, left, right, hb, ring, c++, slot, t, Tp, a.err);
            slot = (slot + 1 == S) ? 0 : slot + 1;
#pragma unroll
            for (int r = 0; r < PR; ++r)
#pragma unroll
                for (int j = 0; j < E; ++j) { acc[r][j] += k[r][j]; dx[r][j] = fmaf(h6, acc[r][j], dx[r][j]); }
        }
        if (a.mode == 2) {
            ring.drain(a.err);
            __syncthreads();
            if (tid == 0)
                for (int i = 0; i < S; ++i) mbar_inval(ring.bar0 + 8u * i);
            return;
        }
        __syncthreads();   // last tangent-linear stage read before the adjoint refills its buffer
    }

    float lam[PR][E];
#pragma unroll
    for (int r = 0; r < PR; ++r)
#pragma unroll
        for (int j = 0; j < E; ++j) lam[r][j] = 0.f;
    for (int tt = a.T;; --tt) {
        const int o0 = a.optr[tt], o1 = a.optr[tt + 1];
        if (o0 < o1) {
            if (live)
#pragma unroll
                for (int r = 0; r < PR; ++r) {
                    float *st = state + (g * PR + r) * SP;
#pragma unroll
                    for (int j = 0; j < E; ++j) st[swz(tE + j)] = lam[r][j];
                }
            __syncthreads();
#pragma unroll
            for (int r = 0; r < PR; ++r) {
                const int probe = probe0 + r;
                if (live && probe < a.ncols) {
                    float *st = state + (g * PR + r) * SP;
                    const float *rr = a.r + (size_t)probe * (size_t)a.p;
                    for (int o = o0 + t; o < o1; o += Tp) atomicAdd(&st[swz(a.oslot[o])], rr[o]);
                }
            }
            __syncthreads();
#pragma unroll
            for (int r = 0; r < PR; ++r) {
                const float *st = state + (g * PR + r) * SP;
#pragma unroll
                for (int j = 0; j < E; ++j) lam[r][j] = (j < len) ? st[swz(tE + j)] : 0.f;
            }
        }
        if (tt == 0) break;
        float lk[PR][E], ls[PR][E], lx[PR][E];
#pragma unroll
        for (int r = 0; r < PR; ++r)
#pragma unroll
            for (int j = 0; j < E; ++j) lk[r][j] = h6 * lam[r][j];
        ad_stage<E, PR>(lk, ls, full, H, nthr, tid, left, right, hb, ring, c++, slot, t, Tp, offL, oddL, tr, a.err);
        slot = (slot + 1 == S) ? 0 : slot + 1;
#pragma unroll
        for (int r = 0; r < PR; ++r)
#pragma unroll
            for (int j = 0; j < E; ++j) { lx[r][j] = lam[r][j] + ls[r][j]; lk[r][j] = fmaf(h3, lam[r][j], h * ls[r][j]); }
        ad_stage<E, PR>(lk, ls, full, H, nthr, tid, left, right, hb, ring, c++, slot, t, Tp, offL, oddL, tr, a.err);
        slot = (slot + 1 == S) ? 0 : slot + 1;
#pragma unroll
        for (int r = 0; r < PR; ++r)
#pragma unroll
            for (int j = 0; j < E; ++j) { lx[r][j] += ls[r][j]; lk[r][j] = fmaf(h3, lam[r][j], h2 * ls[r][j]); }
        ad_stage<E, PR>(lk, ls, full, H, nthr, tid, left, right, hb, ring, c++, slot, t, Tp, offL, oddL, tr, a.err);
        slot = (slot + 1 == S) ? 0 : slot + 1;
#pragma unroll
        for (int r = 0; r < PR; ++r)
#pragma unroll
            for (int j = 0; j < E; ++j) { lx[r][j] += ls[r][j]; lk[r][j] = fmaf(h6, lam[r][j], h2 * ls[r][j]); }
        ad_stage<E, PR>(lk, ls, full, H, nthr, tid, left, right, hb, ring, c++, slot, t, Tp, offL, oddL, tr, a.err);
        slot = (slot + 1 == S) ? 0 : slot + 1;
#pragma unroll
        for (int r = 0; r < PR; ++r)
#pragma unroll
            for (int j = 0; j < E; ++j) lam[r][j] = lx[r][j] + ls[r][j];
    }

    ring.drain(a.err);
    __syncthreads();
    if (tid == 0)
        for (int i = 0; i < S; ++i) mbar_inval(ring.bar0 + 8u * i);
    if (live)
#pragma unroll
        for (int r = 0; r < PR; ++r) {
            float *st = state + (g * PR + r) * SP;
#pragma unroll
            for (int j = 0; j < E; ++j)
                if (j < len) st[swz(s0 + j)] = a.sig[s0 + j] * lam[r][j];
        }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < PR; ++r) {
        const int probe = probe0 + r;
        float y[E];
        band_apply_t<E>(state + (g * PR + r) * SP, a.band, a.hl, a.hh, n, s0, len, y);
        if (live && probe < a.ncols) {
            float *yo = a.Y + (size_t)probe * a.ld;
            const float *w = a.W ? a.W + (size_t)probe * a.ld : nullptr;
#pragma unroll
            for (int j = 0; j < E; ++j)
                if (j < len) yo[s0 + j] = y[j] + ((a.add_identity && w) ? w[s0 + j] : 0.f);
        }
    }
}

template <int E, int PR, int MAXT, bool RAGGED, int MINB = 1>
__global__ void __launch_bounds__(MAXT, MINB) l96_hvp_tma_kernel(const TmaArgs a)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ int abort_flag;
    if (threadIdx.x == 0) abort_flag = 0;
    hvp_tma_body<E, PR, RAGGED>(a, blockIdx.x, smem_raw, &abort_flag);
}

// Persistent kernel over a queue of (window, block) items of several
// Lorenz-96 windows: each CTA takes the next item until the queue is empty,
// so windows of different sizes share one launch.
struct BatchItem {
    int win, blk;
};

template <int MAXT>
__global__ void __launch_bounds__(MAXT, 1) l96_hvp_batch_kernel(const TmaArgs *args, const BatchItem *items, int nitems,
                                                                int *counter)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ int abort_flag, item_s;
    if (threadIdx.x == 0) abort_flag = 0;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) item_s = atomicAdd(counter, 1);
        __syncthreads();
        const int it = item_s;
        if (it >= nitems) break;
        const BatchItem bi = items[it];
        const TmaArgs a = args[bi.win];
        if (a.geom.E == 4) hvp_tma_body<4, 2>(a, bi.blk, smem_raw, &abort_flag);
        else if (a.geom.E == 8) hvp_tma_body<8, 2>(a, bi.blk, smem_raw, &abort_flag);
        else hvp_tma_body<16, 1>(a, bi.blk, smem_raw, &abort_flag);
    }
}


// Shared memory: barriers, S stage buffers, halo (2 buffers x 3 x PR x nthr),
// state copies of the P * PR probes.
size_t tma_smem_bytes(int Np, int nthr, int P, int S, int PR)
{
    return 128 + (size_t)S * Np * 8 + sizeof(float) * (6 * (size_t)PR * nthr + (size_t)P * PR * stage_pad_t(Np));
}

}  // namespace

// Choose P thread groups per CTA and ring depth S for the shared-memory
// budget; positive hints are taken when they fit.
static bool tma_plan(const ChunkGeom &g, int ncols, int PR, int maxthr, size_t smem_max, int P_hint, int S_hint,
                     int *P_out, int *S_out)
{
    const int groups_needed = (ncols + PR - 1) / PR;
    int Pmax = maxthr / g.Tp;
    if (Pmax > 64) Pmax = 64;
    if (Pmax > groups_needed) Pmax = groups_needed;
    if (P_hint > 0 || S_hint > 0) {
        const int P = (P_hint > 0 && P_hint <= Pmax) ? P_hint : Pmax;
        const int S = (S_hint >= 2 && S_hint <= 8) ? S_hint : 4;
        if (P >= 1 && tma_smem_bytes(g.Np, P * g.Tp, P, S, PR) <= smem_max) {
            *P_out = P;
            *S_out = S;
            return true;
        }
    }
    for (int P = Pmax; P >= 1; --P)
        for (int S = 4; S >= 2; --S)
            if (tma_smem_bytes(g.Np, P * g.Tp, P, S, PR) <= smem_max) {
                *P_out = P;
                *S_out = S;
                return true;
            }
    return false;
}

template <int E, int PR, int MAXT, int MINB = 1>
static cudaError_t launch_tma(const TmaArgs &a, int grid, int nthr, size_t sm, cudaStream_t s)
{
    const bool ragged = a.geom.g != 0;
    auto kern = ragged ? l96_hvp_tma_kernel<E, PR, MAXT, true, MINB> : l96_hvp_tma_kernel<E, PR, MAXT, false, MINB>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    count_launch();
    kern<<<grid, nthr, sm, s>>>(a);
    return cudaGetLastError();
}

cudaError_t l96_hvp_tma_launch(const L96Dev &m, const float2 *coef, const float *W, float *Y, int64_t ld, int ncols,
                               int add_identity, float *r, int mode, int *err, cudaStream_t s, int P_hint, int S_hint,
                               int wait_polls, bool two_per_sm)
{
    if (ncols <= 0) return cudaSuccess;
    int dev = 0, smem_optin = 0, smem_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    const int E = m.geom.E;
    // two probes per thread (registers) for E <= 8: 512-thread CTAs, one per SM; two_per_sm
    // (E = 8): one probe per thread in 64 registers, two CTAs per SM sharing its shared memory
    const bool pair = two_per_sm && E == 8;
    const int PR = (E <= 8 && !pair) ? 2 : 1;
    const int maxthr = 512;
    const size_t smem_max = pair ? (size_t)smem_sm / 2 - 1024 : (size_t)smem_optin - 1024;
    int P = 1, S = 2;
    if (!tma_plan(m.geom, ncols, PR, maxthr, smem_max, P_hint, S_hint, &P, &S))
        return cudaErrorInvalidConfiguration;
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
    a.wait_polls = wait_polls >= 0 ? wait_polls : kWaitPolls;
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
    const size_t sm = tma_smem_bytes(m.geom.Np, nthr, P, S, PR);
    const int per_cta = P * PR;
    const int grid = (ncols + per_cta - 1) / per_cta;
    switch (E) {
    case 4: return launch_tma<4, 2, 512>(a, grid, nthr, sm, s);
    case 8: return pair ? launch_tma<8, 1, 512, 2>(a, grid, nthr, sm, s) : launch_tma<8, 2, 512>(a, grid, nthr, sm, s);
    case 16: return launch_tma<16, 1, 512>(a, grid, nthr, sm, s);
    default: return cudaErrorInvalidValue;
    }
}

// ---------------------------------------------------------------------------
// Batch of windows in one persistent launch
// ---------------------------------------------------------------------------
void hvp_batch_free(HvpBatchPlan *plan)
{
    if (!plan) return;
    cudaFree(plan->d_args);
    cudaFree(plan->d_items);
    cudaFree(plan->d_counter);
    plan->d_args = plan->d_items = nullptr;
    plan->d_counter = nullptr;
    plan->nitems = plan->nwin = 0;
}

cudaError_t hvp_batch_plan(const HvpBatchWindow *w, int nwin, int P_cap, int S_req, HvpBatchPlan *plan)
{
    constexpr int kThreads = 512;
    int dev = 0, smem_optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const size_t smax = (size_t)smem_optin - 1024;
    std::vector<TmaArgs> args(nwin);
    struct Cand {
        double cost;
        BatchItem it;
    };
    std::vector<Cand> items;
    size_t smem = 0;
    for (int i = 0; i < nwin; ++i) {
        const L96Dev &m = *w[i].m;
        const ChunkGeom &g = m.geom;
        const int PR = (g.E <= 8) ? 2 : 1;
        if (g.Tp > kThreads || w[i].ncols < 1) return cudaErrorInvalidConfiguration;
        int P = kThreads / g.Tp;
        if (P > 64) P = 64;
        if (P_cap > 0 && P > P_cap) P = P_cap;
        const int groups = (w[i].ncols + PR - 1) / PR;
        if (P > groups) P = groups;
        int S = (S_req >= 2 && S_req <= 8) ? S_req : 4;
        while (S > 2 && tma_smem_bytes(g.Np, kThreads, P, S, PR) > smax) --S;
        while (P > 1 && tma_smem_bytes(g.Np, kThreads, P, S, PR) > smax) --P;
        const size_t sm = tma_smem_bytes(g.Np, kThreads, P, S, PR);
        if (sm > smax) return cudaErrorInvalidConfiguration;
        if (sm > smem) smem = sm;
        TmaArgs &a = args[i];
        a.geom = g;
        a.T = m.T;
        a.P = P;
        a.S = S;
        a.p = m.p;
        a.hl = m.band.hl;
        a.hh = m.band.hh;
        a.ncols = w[i].ncols;
        a.add_identity = 0;
        a.mode = 0;
        a.wait_polls = kWaitPolls;
        a.dt = (float)m.dt;
        a.coef = w[i].coef;
        a.optr = m.optr;
        a.oslot = m.oslot;
        a.rinv = m.rinv32;
        a.band = m.band32;
        a.sig = m.sig32;
        a.W = w[i].W;
        a.Y = w[i].Y;
        a.r = w[i].r;
        a.ld = w[i].ld;
        a.err = w[i].err;
        const int nblk = (w[i].ncols + P * PR - 1) / (P * PR);
        // per-thread work of an item grows with T * E * PR: longest first
        const double cost = (double)m.T * g.E * PR;
        for (int b = 0; b < nblk; ++b) items.push_back({cost, {i, b}});
    }
    std::stable_sort(items.begin(), items.end(), [](const Cand &x, const Cand &y) { return x.cost > y.cost; });
    std::vector<BatchItem> its(items.size());
    for (size_t i = 0; i < items.size(); ++i) its[i] = items[i].it;
    hvp_batch_free(plan);
    cudaError_t e;
    if ((e = cudaMalloc(&plan->d_args, sizeof(TmaArgs) * nwin)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&plan->d_items, sizeof(BatchItem) * its.size())) != cudaSuccess) return e;
    if ((e = cudaMalloc(&plan->d_counter, sizeof(int))) != cudaSuccess) return e;
    if ((e = cudaMemcpy(plan->d_args, args.data(), sizeof(TmaArgs) * nwin, cudaMemcpyHostToDevice)) != cudaSuccess)
        return e;
    if ((e = cudaMemcpy(plan->d_items, its.data(), sizeof(BatchItem) * its.size(), cudaMemcpyHostToDevice)) !=
        cudaSuccess)
        return e;
    // a copy from pageable memory may still be in flight when cudaMemcpy returns, and the batch
    // kernel runs on streams that do not wait for the legacy stream: finish it here
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(l96_hvp_batch_kernel<kThreads>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem)) != cudaSuccess)
        return e;
    plan->nwin = nwin;
    plan->nitems = (int)its.size();
    plan->nthr = kThreads;
    plan->smem = smem;
    plan->grid = plan->nitems < num_sms() ? plan->nitems : num_sms();
    plan->P_cap = P_cap;
    plan->S = S_req;
    return cudaSuccess;
}

cudaError_t hvp_batch_launch(const HvpBatchPlan &plan, cudaStream_t s)
{
    if (plan.nitems == 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(plan.d_counter, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    count_launch();
    l96_hvp_batch_kernel<512><<<plan.grid, plan.nthr, plan.smem, s>>>(
        (const TmaArgs *)plan.d_args, (const BatchItem *)plan.d_items, plan.nitems, plan.d_counter);
    return cudaGetLastError();
}

}  // namespace riot
