// FP32 batched Lorenz-96 Hessian-vector kernel, warp-synchronous.
//
// The same mathematics as l96_hvp_kernel and l96_hvp_tma_kernel (Eq. 4: for every
// sketch column one tangent-linear RK4 integration forward and one adjoint
// integration backward along the stored trajectory, Algorithm 3's parallel loop),
// arranged so that no stage needs a CTA-wide barrier:
//  * A CTA holds the whole state of PR probes: thread t keeps E consecutive
//    variables (chunk t of the ring of n variables) of each probe in registers.
//  * The periodic stencil's neighbours (i-2, i-1, i+1) cross chunk boundaries
//    through a double-buffered shared-memory halo (each thread publishes the three
//    values its neighbours need), or (SHFL) by warp shuffles between the lanes of a
//    warp, only the two edge lanes of a warp publishing theirs for the neighbouring
//    warps.  Instead of a CTA-wide barrier per stage, a warp meets only its two
//    neighbouring warps, at a hardware named barrier per pair, and only after it has
//    computed the elements of its chunks that need no value of another thread.
//  * Every warp streams the stage coefficients (a, b) = (X_{i-1}, X_{i+1} - X_{i-2})
//    of its own chunks, plus one pair of each neighbouring warp, from a per-warp
//    contiguous block of global memory into its own ring of S shared-memory
//    slots by 1-D TMA (cp.async.bulk, completion on an mbarrier per slot).  The
//    warp refills a slot itself once its lanes are past it: no producer thread
//    and no cross-warp dependence for the coefficients.
//  * Observations are sorted by (step, slot), with a table of each thread's
//    range per observed step, so the thread that owns a variable writes its
//    residual in the forward pass and adds its forcing in the backward pass.
//  * The adjoint tendency J^T m is formed with three FMAs per variable.
// Every wait on a copy is bounded; one that runs out raises a CTA-wide abort flag and
// the error flag, later waits return at once, and before the CTA exits each warp waits
// (full bound) for every copy it started.  The named barriers need no bound: every warp
// passes the same sequence of them whatever the data or an abort.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "internal.h"

namespace riot {

namespace {

// A wait gives up after kWaitNs of global time (or after the test limit of tries).
constexpr unsigned long long kWaitNs = 500000000ull;   // 0.5 s


__device__ __forceinline__ int swzw(int x) { return x + (x >> 3); }
__host__ __device__ __forceinline__ int pad_state(int Np) { return Np + (Np >> 3) + 2; }

__device__ __forceinline__ uint32_t saddr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init_w(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_inval_w(uint32_t bar)
{
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_arrive_w(uint32_t bar)
{
    asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_test_w(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for the completion of the phase of parity `parity`: at most `tries` tries when
// tries >= 0 (0: give up at once), and never longer than kWaitNs.  After any wait of the
// CTA gave up, returns false at once.
__device__ __forceinline__ bool mbar_wait_w(uint32_t bar, uint32_t parity, int tries, volatile int *abort_flag,
                                            int *err)
{
    if (*abort_flag) return false;
    if (tries != 0) {
        if (mbar_test_w(bar, parity)) return true;
        const unsigned long long t0 = global_ns();
        for (int i = 1; tries < 0 || i < tries; ++i) {
            if (mbar_test_w(bar, parity)) return true;
            if ((i & 63) == 0 && global_ns() - t0 > kWaitNs) break;
        }
    }
    *abort_flag = 1;
    atomicMax(err, 1);
    return false;
}

__device__ __forceinline__ void tma_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar)
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

struct WarpArgs {
    ChunkGeom geom;
    int T, S, p, hl, hh, ncols, add_identity, wait_polls, nwarps, slot4;
    float dt;
    const float4 *coef;   // [4T][nwarps][slot4]
    const int *ostep, *ostart, *oslot, *operm;
    const float *rinv, *band, *sig, *W;
    float *Y, *r;
    long long ld;
    int *err;
};

// Per-warp stream of coefficient slots.  Lane 0 issues the copies and tracks how many
// it started (`issued`) and saw land (`landed`, from its own waits) so that after an
// abort it can wait for the rest before the CTA exits.  The slot and phase parity of the
// current stage are kept incrementally (no division by the run-time ring depth).
struct WarpRing {
    const float4 *src;     // this warp's block of stage 0
    float4 *buf;           // S slots of slot4 float4
    uint32_t bar0;         // S mbarriers
    int S, slot4, total, stride4, polls;   // stride4: float4 between stages of this warp
    int issued, landed;
    int slot;              // slot of the current stage
    uint32_t phase;        // parity of the current stage's phase in its slot
    // stream position c -> stage block: forward through the 4T tangent-linear stages,
    // then backward through them for the adjoint
    __device__ int blk(int c) const { return c < total / 2 ? c : total - 1 - c; }
    __device__ void issue_to(int c, int sl)
    {
        tma_g2s(saddr(buf + (size_t)sl * slot4), src + (size_t)blk(c) * stride4, (uint32_t)slot4 * 16u,
                bar0 + 8u * sl);
        issued = c + 1;
    }
    __device__ bool wait(int c, volatile int *abort_flag, int *err)
    {
        const bool ok = mbar_wait_w(bar0 + 8u * slot, phase, polls, abort_flag, err);
        if (ok && (threadIdx.x & 31) == 0) landed = c + 1;
        return ok;
    }
    __device__ const float4 *cur() const { return buf + (size_t)slot * slot4; }
    // lane 0, after every lane of the warp is done with stage c's slot: refill it with c + S
    __device__ void refill(int c, volatile int *abort_flag)
    {
        if ((threadIdx.x & 31) == 0 && c + S < total && !*abort_flag) issue_to(c + S, slot);
    }
    __device__ void advance()
    {
        if (++slot == S) {
            slot = 0;
            phase ^= 1u;
        }
    }
    // after an abort: wait (full time bound, whatever the test limit) for the copies started
    __device__ void drain(int *err)
    {
        if ((threadIdx.x & 31) != 0) return;
        for (int c = landed; c < issued; ++c) {
            const unsigned long long t0 = global_ns();
            bool done = false;
            while (!done && global_ns() - t0 <= kWaitNs) done = mbar_test_w(bar0 + 8u * (c % S), (uint32_t)((c / S) & 1));
            if (!done) atomicMax(err, 2);
        }
    }
};

// Meeting of a warp with its two neighbouring warps at hardware named barriers, one per
// pair of neighbouring warps (bar.sync id, 64: pair (w, w + 1) uses id w, so up to 16
// warps).  Even warps meet the left neighbour first, odd warps the right one, so the
// pairwise waits never form a cycle; a warp waiting at a named barrier issues nothing.
// Every warp runs the same stages, so every pair barrier is always completed.
__device__ __forceinline__ void meet_neighbours(int w, int wl)
{
    if (w & 1) {
        asm volatile("bar.sync %0, 64;" ::"r"(w) : "memory");
        asm volatile("bar.sync %0, 64;" ::"r"(wl) : "memory");
    } else {
        asm volatile("bar.sync %0, 64;" ::"r"(wl) : "memory");
        asm volatile("bar.sync %0, 64;" ::"r"(w) : "memory");
    }
}

// v[j] for a register array and a run-time j (selects, so v stays in registers)
template <int E>
__device__ __forceinline__ float pick(const float (&v)[E], int j)
{
    float out = 0.f;
#pragma unroll
    for (int jj = 0; jj < E; ++jj) out = (jj == j) ? v[jj] : out;
    return out;
}

template <int E>
__device__ __forceinline__ void band_apply_w(const float *st, const float *band, int hl, int hh, int n, int s0, int len,
                                             float (&out)[E])
{
#pragma unroll
    for (int j = 0; j < E; ++j) out[j] = 0.f;
    for (int d = -hl; d <= hh; ++d) {
        const float wgt = band[d + hl];
#pragma unroll
        for (int j = 0; j < E; ++j) {
            int ii = s0 + j + d;
            ii += (ii < 0) ? n : 0;
            ii -= (ii >= n) ? n : 0;
            if (j < len) out[j] = fmaf(wgt, st[swzw(ii)], out[j]);
        }
    }
}

template <int E, int PR, bool RAGGED, bool SHFL>
__global__ void __launch_bounds__(512, 1) l96_hvp_warp_kernel(const WarpArgs a)
{
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ int abort_flag;
    const ChunkGeom &G = a.geom;
    const int n = G.n, Tp = G.Tp, NW = a.nwarps, S = a.S;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const bool live = tid < Tp;
    const int t = live ? tid : Tp - 1;
    const int rlane = (w == NW - 1) ? (Tp - 1 - 32 * w) : 31;   // last live lane of this warp
    const int s0 = G.start(t), len = G.len(t);
    const bool full = !RAGGED || len == E;
    const int tl = (t == 0) ? Tp - 1 : t - 1;
    const int lenL = G.len(tl);
    const int pairL = (lenL - 1) >> 1, oddL = (lenL - 1) & 1;
    const int probe0 = blockIdx.x * PR;
    const float h = a.dt, h2 = 0.5f * a.dt, h6 = a.dt / 6.f, h3 = a.dt / 3.f;

    uint64_t *bars = reinterpret_cast<uint64_t *>(smem);                 // NW*S ring + 1 end barrier
    const size_t bar_bytes = (((size_t)NW * S + 1) * 8 + 127) & ~(size_t)127;
    float4 *ringbuf = reinterpret_cast<float4 *>(smem + bar_bytes);     // NW * S * slot4
    // halo: 2 buffers x 3 PR values x every thread (the values its neighbours need)
    float *H = reinterpret_cast<float *>(ringbuf + (size_t)NW * S * a.slot4);
    const int nthr = 32 * NW;
    const int left = (t == 0) ? Tp - 1 : t - 1, right = (t == Tp - 1) ? 0 : t + 1;
    const int wl = (w == 0) ? NW - 1 : w - 1;
    float *state = reinterpret_cast<float *>(ringbuf);                  // aliases the ring (prologue, epilogue)
    const int SP = pad_state(G.Np);

    WarpRing ring;
    ring.src = a.coef + (size_t)w * a.slot4;
    ring.buf = ringbuf + (size_t)w * S * a.slot4;
    ring.bar0 = saddr(bars + (size_t)w * S);
    ring.S = S;
    ring.slot4 = a.slot4;
    ring.total = 8 * a.T;
    ring.stride4 = NW * a.slot4;
    ring.polls = a.wait_polls;
    ring.issued = 0;
    ring.landed = 0;
    ring.slot = 0;
    ring.phase = 0;

    const uint32_t end_bar = saddr(bars + (size_t)NW * S);   // all warps past the main loop

    if (tid == 0) abort_flag = 0;
    if (lane == 0) {
        for (int i = 0; i < S; ++i) mbar_init_w(ring.bar0 + 8u * i, 1);
        if (w == 0) mbar_init_w(end_bar, NW);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }

    // ---- prologue: dx = L w for the PR probes (state copies in the ring's memory) ----
#pragma unroll
    for (int r = 0; r < PR; ++r) {
        const int probe = probe0 + r;
        const bool active = probe < a.ncols;
        const float *wcol = a.W + (size_t)(active ? probe : 0) * a.ld;
        float *st = state + (size_t)r * SP;
        for (int i = tid; i < n; i += blockDim.x) st[swzw(i)] = active ? wcol[i] : 0.f;
    }
    __syncthreads();
    float dx[PR][E];
#pragma unroll
    for (int r = 0; r < PR; ++r) {
        float tmp[E];
        band_apply_w<E>(state + (size_t)r * SP, a.band, a.hl, a.hh, n, s0, len, tmp);
#pragma unroll
        for (int j = 0; j < E; ++j) dx[r][j] = (j < len) ? tmp[j] * a.sig[s0 + (j < len ? j : 0)] : 0.f;
    }
    __syncthreads();   // the ring may now overwrite the state copies
    if (lane == 0)
        for (int c = 0; c < S && c < ring.total; ++c) ring.issue_to(c, c);

    volatile int *abort_v = &abort_flag;
    int *err = a.err;
    int c = 0;   // stage position in the coefficient stream (TL stages 0..4T-1, then AD)

    // ---------------------------------------------------------------- tangent linear
    for (int tt = 0;; ++tt) {
        const int k = a.ostep[tt];
        if (k >= 0 && live) {
            const int *os = a.ostart + (size_t)k * (Tp + 1);
            const int ob = os[t], oe = os[t + 1];
            for (int o = ob; o < oe; ++o) {
                const int j = a.oslot[o] - t * E;
                const float ri = a.rinv[a.operm[o]];
#pragma unroll
                for (int r = 0; r < PR; ++r)
                    if (probe0 + r < a.ncols) a.r[(size_t)(probe0 + r) * a.p + o] = ri * pick<E>(dx[r], j);
            }
        }
        if (tt == a.T) break;
        float s[PR][E], acc[PR][E];
#pragma unroll
        for (int r = 0; r < PR; ++r)
#pragma unroll
            for (int j = 0; j < E; ++j) {
                s[r][j] = dx[r][j];
                acc[r][j] = 0.f;
            }
#pragma unroll 1
        for (int stg = 0; stg < 4; ++stg, ++c, ring.advance()) {
            // the values the neighbouring threads need (last two valid, first): published in
            // shared memory (SHFL: shuffled inside the warp, published by the two edge lanes only)
            float *Hb = H + (size_t)(c & 1) * 3 * PR * nthr;
            float v0[PR], v1[PR], v2[PR];
#pragma unroll
            for (int r = 0; r < PR; ++r) {
                v0[r] = full ? s[r][E - 2] : s[r][E - 3];
                v1[r] = full ? s[r][E - 1] : s[r][E - 2];
                v2[r] = s[r][0];
                if (!SHFL || lane == 0 || lane == rlane) {
                    Hb[(0 * PR + r) * nthr + tid] = v0[r];
                    Hb[(1 * PR + r) * nthr + tid] = v1[r];
                    Hb[(2 * PR + r) * nthr + tid] = v2[r];
                }
            }
            float m2[PR], m1[PR], p1[PR];
            ring.wait(c, abort_v, err);
            const float4 *cf = ring.cur() + lane;
            float ca[E], cb[E];
#pragma unroll
            for (int j2 = 0; j2 < E / 2; ++j2) {
                const float4 cc = cf[j2 * 32];
                ca[2 * j2] = cc.x;
                cb[2 * j2] = cc.y;
                ca[2 * j2 + 1] = cc.z;
                cb[2 * j2 + 1] = cc.w;
            }
            __syncwarp();
            ring.refill(c, abort_v);   // the coefficients are in registers: refill the slot now
            float kk[PR][E];
            // interior elements first (no value of another warp needed) ...
#pragma unroll
            for (int j = 2; j <= E - 3; ++j)
#pragma unroll
                for (int r = 0; r < PR; ++r)
                    kk[r][j] = fmaf(ca[j], s[r][j + 1] - s[r][j - 2], fmaf(cb[j], s[r][j - 1], -s[r][j]));
            // ... then the neighbours' values from shared memory behind the pair barriers
            // (SHFL: shuffles inside the warp, shared memory for the edge lanes only: lane 0
            // from the warp before, the last live lane from the warp after)
            if constexpr (SHFL) {
#pragma unroll
                for (int r = 0; r < PR; ++r) {
                    m2[r] = __shfl_up_sync(0xffffffffu, v0[r], 1);
                    m1[r] = __shfl_up_sync(0xffffffffu, v1[r], 1);
                    p1[r] = __shfl_down_sync(0xffffffffu, v2[r], 1);
                }
            }
            meet_neighbours(w, wl);
#pragma unroll
            for (int r = 0; r < PR; ++r) {
                if (!SHFL || lane == 0) {
                    m2[r] = Hb[(0 * PR + r) * nthr + left];
                    m1[r] = Hb[(1 * PR + r) * nthr + left];
                }
                if (!SHFL || lane >= rlane) p1[r] = Hb[(2 * PR + r) * nthr + right];
            }
#pragma unroll
            for (int j = 0; j < E; ++j) {
                if (j >= 2 && j <= E - 3) continue;
#pragma unroll
                for (int r = 0; r < PR; ++r) {
                    const float xm2 = (j == 0) ? m2[r] : (j == 1 ? m1[r] : s[r][j >= 2 ? j - 2 : 0]);
                    const float xm1 = (j == 0) ? m1[r] : s[r][j >= 1 ? j - 1 : 0];
                    float xp1;
                    if (j == E - 1) xp1 = p1[r];
                    else if (j == E - 2) xp1 = full ? s[r][E - 1] : p1[r];
                    else xp1 = s[r][j + 1 < E ? j + 1 : 0];
                    kk[r][j] = fmaf(ca[j], xp1 - xm2, fmaf(cb[j], xm1, -s[r][j]));
                }
            }
            if (RAGGED && !full)
#pragma unroll
                for (int r = 0; r < PR; ++r) kk[r][E - 1] = 0.f;
            // RK4 combination with stage-uniform weights (no per-element selects): acc gathers
            // k1 + 2 k2 + 2 k3 + k4, s is the next stage's input dx + c k
            const float wgt = (stg == 1 || stg == 2) ? 2.f : 1.f;
            const float cs = (stg == 2) ? h : h2;
#pragma unroll
            for (int r = 0; r < PR; ++r)
#pragma unroll
                for (int j = 0; j < E; ++j) {
                    acc[r][j] = fmaf(wgt, kk[r][j], acc[r][j]);
                    s[r][j] = fmaf(cs, kk[r][j], dx[r][j]);
                }
        }
#pragma unroll
        for (int r = 0; r < PR; ++r)
#pragma unroll
            for (int j = 0; j < E; ++j) dx[r][j] = fmaf(h6, acc[r][j], dx[r][j]);
    }

    // ---------------------------------------------------------------- adjoint
    float lam[PR][E];
#pragma unroll
    for (int r = 0; r < PR; ++r)
#pragma unroll
        for (int j = 0; j < E; ++j) lam[r][j] = 0.f;
    const int cl_idx = (lane == 0) ? (E / 2) * 32 : pairL * 32 + lane - 1;
    const int cr_idx = (lane == rlane) ? (E / 2) * 32 + 1 : lane + 1;
    for (int tt = a.T;; --tt) {
        const int k = a.ostep[tt];
        if (k >= 0 && live) {
            const int *os = a.ostart + (size_t)k * (Tp + 1);
            const int ob = os[t], oe = os[t + 1];
            for (int o = ob; o < oe; ++o) {
                const int j = a.oslot[o] - t * E;
#pragma unroll
                for (int r = 0; r < PR; ++r) {
                    const float v = (probe0 + r < a.ncols) ? a.r[(size_t)(probe0 + r) * a.p + o] : 0.f;
#pragma unroll
                    for (int jj = 0; jj < E; ++jj) lam[r][jj] += (jj == j) ? v : 0.f;
                }
            }
        }
        if (tt == 0) break;
        float lx[PR][E], lk[PR][E];
#pragma unroll
        for (int r = 0; r < PR; ++r)
#pragma unroll
            for (int j = 0; j < E; ++j) {
                lk[r][j] = h6 * lam[r][j];
                lx[r][j] = lam[r][j];
            }
#pragma unroll 1
        for (int stg = 0; stg < 4; ++stg, ++c, ring.advance()) {
            float *Hb = H + (size_t)(c & 1) * 3 * PR * nthr;
            float u0[PR], u1[PR], u2[PR];
#pragma unroll
            for (int r = 0; r < PR; ++r) {
                u0[r] = full ? lk[r][E - 1] : lk[r][E - 2];
                u1[r] = lk[r][0];
                u2[r] = lk[r][1];
                if (!SHFL || lane == 0 || lane == rlane) {
                    Hb[(0 * PR + r) * nthr + tid] = u0[r];
                    Hb[(1 * PR + r) * nthr + tid] = u1[r];
                    Hb[(2 * PR + r) * nthr + tid] = u2[r];
                }
            }
            float mL[PR], mR0[PR], mR1[PR];
            ring.wait(c, abort_v, err);
            const float4 *sl = ring.cur();
            const float4 *cf = sl + lane;
            const float4 cl = sl[cl_idx], cr = sl[cr_idx];
            const float aL = oddL ? cl.z : cl.x;
            float ca[E], cb[E];
#pragma unroll
            for (int j2 = 0; j2 < E / 2; ++j2) {
                const float4 cc = cf[j2 * 32];
                ca[2 * j2] = cc.x;
                cb[2 * j2] = cc.y;
                ca[2 * j2 + 1] = cc.z;
                cb[2 * j2 + 1] = cc.w;
            }
            __syncwarp();
            ring.refill(c, abort_v);
            // (J^T m)_j = a_{j-1} m_{j-1} - a_{j+2} m_{j+2} + b_{j+1} m_{j+1} - m_j:
            // interior elements (all three neighbours in this chunk, also a short one) first
            float ls[PR][E];
#pragma unroll
            for (int j = 1; j <= E - 4; ++j)
#pragma unroll
                for (int r = 0; r < PR; ++r)
                    ls[r][j] = fmaf(ca[j - 1], lk[r][j - 1],
                                    fmaf(-ca[j + 2], lk[r][j + 2], fmaf(cb[j + 1], lk[r][j + 1], -lk[r][j])));
            if constexpr (SHFL) {
#pragma unroll
                for (int r = 0; r < PR; ++r) {
                    mL[r] = __shfl_up_sync(0xffffffffu, u0[r], 1);
                    mR0[r] = __shfl_down_sync(0xffffffffu, u1[r], 1);
                    mR1[r] = __shfl_down_sync(0xffffffffu, u2[r], 1);
                }
            }
            meet_neighbours(w, wl);
#pragma unroll
            for (int r = 0; r < PR; ++r) {
                if (!SHFL || lane == 0) mL[r] = Hb[(0 * PR + r) * nthr + left];
                if (!SHFL || lane >= rlane) {
                    mR0[r] = Hb[(1 * PR + r) * nthr + right];
                    mR1[r] = Hb[(2 * PR + r) * nthr + right];
                }
            }
#pragma unroll
            for (int r = 0; r < PR; ++r) {
#pragma unroll
                for (int j = 0; j < E; ++j) {
                    if (j >= 1 && j <= E - 4) continue;
                    // m_{j-1} with a_{j-1}
                    const float mm1 = (j == 0) ? mL[r] : lk[r][j >= 1 ? j - 1 : 0];
                    const float am1 = (j == 0) ? aL : ca[j >= 1 ? j - 1 : 0];
                    // m_{j+1} with b_{j+1}
                    float mp1, bp1;
                    if (j <= E - 2 && (full || j <= E - 3)) {
                        mp1 = lk[r][j + 1 < E ? j + 1 : 0];
                        bp1 = cb[j + 1 < E ? j + 1 : 0];
                    } else {
                        mp1 = mR0[r];
                        bp1 = cr.y;
                    }
                    // m_{j+2} with a_{j+2}
                    float mp2, ap2;
                    if (j <= E - 3 && (full || j <= E - 4)) {
                        mp2 = lk[r][j + 2 < E ? j + 2 : 0];
                        ap2 = ca[j + 2 < E ? j + 2 : 0];
                    } else if (full ? (j == E - 2) : (j == E - 3)) {
                        mp2 = mR0[r];
                        ap2 = cr.x;
                    } else {
                        mp2 = mR1[r];
                        ap2 = cr.z;
                    }
                    ls[r][j] = fmaf(am1, mm1, fmaf(-ap2, mp2, fmaf(bp1, mp1, -lk[r][j])));
                }
                if (RAGGED && !full) ls[r][E - 1] = 0.f;
            }
            // RK4 adjoint stage combination with stage-uniform weights: lx gathers lam plus the
            // four stage outputs; the next stage's input is alpha lam + beta ls with
            // (alpha, beta) = (h/3, h), (h/3, h/2), (h/6, h/2) after stages 1, 2, 3
#pragma unroll
            for (int r = 0; r < PR; ++r)
#pragma unroll
                for (int j = 0; j < E; ++j) lx[r][j] += ls[r][j];
            if (stg < 3) {
                const float al = (stg == 2) ? h6 : h3, be = (stg == 0) ? h : h2;
#pragma unroll
                for (int r = 0; r < PR; ++r)
#pragma unroll
                    for (int j = 0; j < E; ++j) lk[r][j] = fmaf(al, lam[r][j], be * ls[r][j]);
            }
        }
#pragma unroll
        for (int r = 0; r < PR; ++r)
#pragma unroll
            for (int j = 0; j < E; ++j) lam[r][j] = lx[r][j];
    }

    ring.drain(err);
    // CTA-wide meeting point after the main loop, on an mbarrier: named barrier 0 may still be
    // in use by a pair of warps, so __syncthreads must wait until every warp is past the loop
    __syncwarp();
    if (lane == 0) mbar_arrive_w(end_bar);
    {
        const unsigned long long t0 = global_ns();
        while (!mbar_test_w(end_bar, 0) && global_ns() - t0 <= kWaitNs) {
        }
    }
    __syncthreads();   // every warp is past its last wait: barriers and ring memory are free
    if (lane == 0) {
        for (int i = 0; i < S; ++i) mbar_inval_w(ring.bar0 + 8u * i);
    }
    // ---- epilogue: Y = L^T (sigma lam) (+ W) ----
    if (live)
#pragma unroll
        for (int r = 0; r < PR; ++r) {
            float *st = state + (size_t)r * SP;
#pragma unroll
            for (int j = 0; j < E; ++j)
                if (j < len) st[swzw(s0 + j)] = a.sig[s0 + j] * lam[r][j];
        }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < PR; ++r) {
        const int probe = probe0 + r;
        float y[E];
        band_apply_w<E>(state + (size_t)r * SP, a.band, a.hl, a.hh, n, s0, len, y);
        if (live && probe < a.ncols) {
            float *yo = a.Y + (size_t)probe * a.ld;
            const float *wv = a.W + (size_t)probe * a.ld;
#pragma unroll
            for (int j = 0; j < E; ++j)
                if (j < len) yo[s0 + j] = y[j] + (a.add_identity ? wv[s0 + j] : 0.f);
        }
    }
}

// coefw[(stage * NW + w) * slot4 + q] from the FP64 stage coefficients (double2 by slot,
// [4T][Np]): q < E/2 * 32 is pair q / 32 of lane q % 32's chunk; q = E/2 * 32 is the left
// neighbour's last pair, q + 1 the right neighbour's first pair.
__global__ void coef_warp_kernel(const double2 *coef64, ChunkGeom G, int NW, int slot4, long long total,
                                 float4 *out)
{
    const long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (id >= total) return;
    const int q = (int)(id % slot4);
    const long long sw = id / slot4;
    const int w = (int)(sw % NW);
    const long long stage = sw / NW;
    const int E = G.E, Tp = G.Tp;
    const double2 *cs = coef64 + stage * G.Np;
    int t, pair;
    bool valid = true;
    if (q < (E / 2) * 32) {
        t = 32 * w + (q & 31);
        pair = q >> 5;
        valid = t < Tp;
    } else if (q == (E / 2) * 32) {
        t = (32 * w - 1 + Tp) % Tp;
        pair = (G.len(t) - 1) >> 1;
    } else {
        const int live = min(32, Tp - 32 * w);
        t = (32 * w + live) % Tp;
        pair = 0;
    }
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (valid) {
        const double2 c0 = cs[(size_t)t * E + 2 * pair], c1 = cs[(size_t)t * E + 2 * pair + 1];
        v = make_float4((float)c0.x, (float)c0.y, (float)c1.x, (float)c1.y);
    }
    out[id] = v;
}

size_t warp_smem_bytes(int NW, int S, int slot4, int PR, int Np)
{
    const size_t bars = (((size_t)NW * S + 2 * NW) * 8 + 127) & ~(size_t)127;
    size_t ring = (size_t)NW * S * slot4 * 16;
    const size_t state = (size_t)PR * pad_state(Np) * 4;
    if (ring < state) ring = state;
    return bars + ring + (size_t)2 * 3 * PR * 32 * NW * 4;
}

template <int E, int PR, bool RAGGED, bool SHFL>
cudaError_t launch_warp(const WarpArgs &a, int grid, size_t smem, cudaStream_t s)
{
    cudaError_t e = cudaFuncSetAttribute(l96_hvp_warp_kernel<E, PR, RAGGED, SHFL>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    count_launch();
    l96_hvp_warp_kernel<E, PR, RAGGED, SHFL><<<grid, 32 * a.nwarps, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

int warp_probes_per_cta(int E) { return E <= 8 ? 2 : 1; }

bool warp_kernel_fits(const ChunkGeom &g)
{
    return (g.E == 8 || g.E == 16) && g.Tp >= 64 && g.Tp <= 512;
}

cudaError_t l96_warp_tables(const ChunkGeom &g, int T, const std::vector<int> &optr, const std::vector<int> &oslot,
                            std::vector<int> &ostep, std::vector<int> &ostart, std::vector<int> &sslot,
                            std::vector<int> &perm)
{
    const int p = (int)oslot.size();
    ostep.assign(T + 1, -1);
    ostart.clear();
    sslot.resize(p);
    perm.resize(p);
    int nk = 0;
    for (int t = 0; t <= T; ++t) {
        const int o0 = optr[t], o1 = optr[t + 1];
        if (o1 <= o0) continue;
        ostep[t] = nk++;
        std::vector<int> ids(o1 - o0);
        for (int o = o0; o < o1; ++o) ids[o - o0] = o;
        std::stable_sort(ids.begin(), ids.end(), [&](int x, int y) { return oslot[x] < oslot[y]; });
        for (int i = 0; i < o1 - o0; ++i) {
            perm[o0 + i] = ids[i];
            sslot[o0 + i] = oslot[ids[i]];
        }
        // first sorted observation of each thread's chunk (slots t*E .. t*E + E - 1)
        int o = o0;
        for (int th = 0; th <= g.Tp; ++th) {
            while (o < o1 && sslot[o] < th * g.E) ++o;
            ostart.push_back(o);
        }
    }
    if (ostart.empty()) ostart.push_back(0);
    return cudaSuccess;
}

cudaError_t l96_coef_warp(const L96Dev &m, const double2 *coef64, float4 *coefw, cudaStream_t s)
{
    const int NW = (m.geom.Tp + 31) / 32;
    const int slot4 = (m.geom.E / 2) * 32 + 2;
    const long long total = (long long)m.T * 4 * NW * slot4;
    if (total == 0) return cudaSuccess;
    count_launch();
    coef_warp_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(coef64, m.geom, NW, slot4, total, coefw);
    return cudaGetLastError();
}

size_t l96_coef_warp_floats4(const L96Dev &m)
{
    const int NW = (m.geom.Tp + 31) / 32;
    return (size_t)m.T * 4 * NW * ((m.geom.E / 2) * 32 + 2);
}

cudaError_t l96_hvp_warp_launch(const L96Dev &m, const float4 *coefw, const float *W, float *Y, int64_t ld, int ncols,
                                int add_identity, float *r, int *err, cudaStream_t s, int S_hint, int wait_polls,
                                bool shuffle)
{
    if (ncols <= 0) return cudaSuccess;
    if (!warp_kernel_fits(m.geom)) return cudaErrorInvalidConfiguration;
    int dev = 0, smem_optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const int E = m.geom.E, PR = warp_probes_per_cta(E);
    WarpArgs a;
    a.geom = m.geom;
    a.T = m.T;
    a.p = m.p;
    a.hl = m.band.hl;
    a.hh = m.band.hh;
    a.ncols = ncols;
    a.add_identity = add_identity;
    a.wait_polls = wait_polls >= 0 ? wait_polls : -1;
    a.nwarps = (m.geom.Tp + 31) / 32;
    a.slot4 = (E / 2) * 32 + 2;
    a.dt = (float)m.dt;
    a.coef = coefw;
    a.ostep = m.ostep;
    a.ostart = m.ostart;
    a.oslot = m.osslot;
    a.operm = m.osperm;
    a.rinv = m.rinv32;
    a.band = m.band32;
    a.sig = m.sig32;
    a.W = W;
    a.Y = Y;
    a.r = r;
    a.ld = ld;
    a.err = err;
    int S = (S_hint >= 2 && S_hint <= 8) ? S_hint : 8;
    while (S > 2 && warp_smem_bytes(a.nwarps, S, a.slot4, PR, m.geom.Np) > (size_t)smem_optin - 1024) --S;
    const size_t smem = warp_smem_bytes(a.nwarps, S, a.slot4, PR, m.geom.Np);
    if (smem > (size_t)smem_optin - 1024) return cudaErrorInvalidConfiguration;
    a.S = S;
    const int grid = (ncols + PR - 1) / PR;
    const bool ragged = m.geom.g != 0;
    if (shuffle) {
        if (E == 8)
            return ragged ? launch_warp<8, 2, true, true>(a, grid, smem, s) : launch_warp<8, 2, false, true>(a, grid, smem, s);
        return ragged ? launch_warp<16, 1, true, true>(a, grid, smem, s) : launch_warp<16, 1, false, true>(a, grid, smem, s);
    }
    if (E == 8)
        return ragged ? launch_warp<8, 2, true, false>(a, grid, smem, s) : launch_warp<8, 2, false, false>(a, grid, smem, s);
    return ragged ? launch_warp<16, 1, true, false>(a, grid, smem, s) : launch_warp<16, 1, false, false>(a, grid, smem, s);
}

}  // namespace riot
