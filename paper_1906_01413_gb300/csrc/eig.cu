// Symmetric eigendecomposition of the k x k projected matrix K (Algorithm 3:
// K = Z Lambda Z^T) in FP64, laid out for a GPU whose FP64 rate is low per SM:
// every stage spreads its work over all SMs and the number of grid-wide
// synchronisations is O(k), not O(k x sweeps).
//
//  1. Householder tridiagonalisation Q^T K Q = T in one cooperative launch,
//     one grid barrier per column: every CTA derives the next reflector
//     itself, and each warp's rank-2 update of a column is followed at once
//     by that column's product with the next reflector; Q is accumulated as
//     Q^T on the fly.
//  2. T splits where an off-diagonal is negligible; each unreduced block's
//     eigenvalues come from a grid of Sturm counts followed by multisection
//     (one warp per eigenvalue, 32 Sturm counts per round).
//  3. Eigenvectors of T by inverse iteration from distinct pseudo-random
//     starts (tridiagonal LU with partial pivoting, one thread each), then two
//     CholeskyQR passes make them orthonormal (this also separates vectors of
//     eigenvalues that agree to rounding).
//  4. Sort by decreasing eigenvalue, Z = Q Z_T (GEMM).
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <float.h>
#include <math.h>
#include <stdint.h>

#include "fp64_rcp.cuh"
#include "internal.h"

namespace cg = cooperative_groups;

namespace riot {

constexpr int kOctaves = 96;            // pre-bracket grid: |x| = ||T|| 2^(-j/8), j < 8 * kOctaves
constexpr int kGridHalf = 8 * kOctaves;
constexpr int kGrid = 2 * kGridHalf + 3; // negative side, 0, positive side, two outer bounds

size_t eig_work_doubles(int k)
{
    const size_t kk = (size_t)k * k;
    return 9 * kk + 32 * (size_t)k + 1024 + ((size_t)kGrid * k + 1) / 2 + 8 + dinv_doubles(k);
}

namespace {

__device__ __forceinline__ double warp_sum(double v)
{
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

__global__ void eig_init_kernel(const double *K, int k, double *A, double *Qt)
{
    const int64_t total = (int64_t)k * k;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % k), j = (int)(e / k);
        A[e] = 0.5 * (K[i + (int64_t)j * k] + K[j + (int64_t)i * k]);
        Qt[e] = (i == j) ? 1.0 : 0.0;
    }
}

// Block-wide sum of one value per thread (blockDim.x = 256); every thread gets it.  An
// FP64 instruction occupies its sub-partition's FP64 unit for about 64 cycles whatever the
// active lanes, and warps w and w + 4 share a sub-partition: the upper four warps hand their
// values to the lower four, which run one shuffle tree each (one per sub-partition), and one
// thread adds the four partial sums (times `scale`, so that a scaled sum costs the other
// threads nothing).  red: kRedDoubles doubles of shared memory.
constexpr int kRedDoubles = 136;

__device__ __forceinline__ double block_sum(double v, double *red, double scale = 1.0)
{
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    __syncthreads();   // red is free again
    if (wib >= 4) red[threadIdx.x - 128] = v;
    __syncthreads();
    if (wib < 4) {
        v = warp_sum(v + red[threadIdx.x]);
        if (lane == 0) red[128 + wib] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) red[132] = scale * ((red[128] + red[129]) + (red[130] + red[131]));
    __syncthreads();
    return red[132];
}

// Householder reflector of x = col[r0..k-1], computed by the whole CTA (every
// CTA forms the same one): H = I - beta v v^T, H x = e_out e_1; v goes to
// vs[r0..k-1] (zero below r0).  v = x + sign(x0) ||x|| e_1 differs from x in
// one entry, so the scalars (||x||, beta, that entry) are one thread's work and
// the others copy x: FP64 work repeated on every thread costs issue slots of the
// FP64 units that the serial chain waits for.  When x = 0, beta = 0 and H = I
// whatever v holds.
// defer_beta: *beta_out receives the denominator alpha (alpha + |x0|) (0 when x = 0) instead
// of beta, for a caller that forms the reciprocal off the critical path.
__device__ void block_house(const double *col, int k, int r0, double *vs, double *beta_out, double *e_out,
                            double *red, bool defer_beta = false)
{
    double ss = 0.0;
    for (int l = r0 + threadIdx.x; l < k; l += blockDim.x) ss += col[l] * col[l];
    ss = block_sum(ss, red);
    for (int l = threadIdx.x; l < k; l += blockDim.x)
        if (l != r0) vs[l] = (l < r0) ? 0.0 : col[l];
    if (threadIdx.x == 0) {
        const double x0 = col[r0];
        // sqrt(ss) as ss / sqrt(ss): the library rsqrt and one multiplication (about 500
        // cycles against 680 for sqrt on this GPU's FP64 chain)
        const double alpha = (ss > 0.0) ? ss * rsqrt(ss) : 0.0;
        const double sgn = (x0 >= 0.0) ? 1.0 : -1.0;
        vs[r0] = x0 + sgn * alpha;
        const double den = alpha * (alpha + fabs(x0));
        *beta_out = (alpha == 0.0) ? 0.0 : (defer_beta ? den : rcp_fast(den));
        *e_out = (alpha == 0.0) ? 0.0 : -sgn * alpha;
    }
    __syncthreads();
}

// Householder tridiagonalisation Q^T K Q = T, one grid barrier per column.
// Column j: with p = beta A22 v and q = beta Q^T-columns . v of reflector j
// complete, every CTA forms K_ = beta / 2 v^T p, w = p - K_ v, the updated
// column j + 1 and from it reflector j + 1 (the same in every CTA, so nothing
// is exchanged); then each warp updates its A22 or Q^T column (rank 2 or
// rank 1) and at once takes its dot product with reflector j + 1, which is
// the next column's p or q.  Column j + 1 itself is left to the CTAs (each
// derives it), so no CTA writes what another still reads.  p and q are
// double-buffered across the barrier.
// RES (k <= 4 x CTAs): warp w < 4 of CTA b owns column b + G w of A and warp
// 4 + w column b + G w of Q^T (G CTAs) for the whole run, kept in shared memory,
// so each sub-partition carries at most one A column (a rank-2 update, two FMAs
// per row) and one Q^T column (rank 1), and the live A columns (>= j + 1) stay
// spread over the CTAs as j grows; only the column every CTA needs next (j + 2,
// published one step ahead), the last 2 x 2 block and Q^T at the end go back to
// global memory.  Otherwise warps stride over the columns in global memory (L2),
// four loads in flight per lane.
template <bool RES>
__global__ void __launch_bounds__(256) tridiag_kernel(double *A, double *Qt, int k, double *pq, double *d, double *e)
{
    cg::grid_group grid = cg::this_grid();
    extern __shared__ double sm[];
    double *vcur = sm, *vnext = sm + k, *w = sm + 2 * k, *colj = sm + 3 * k, *red = sm + 4 * k;
    double *own = sm + 4 * k + kRedDoubles + (size_t)(threadIdx.x >> 5) * k;   // RES: this warp's column
    __shared__ double bcur_s, bnext_s, enext_s;
    const int lane = threadIdx.x & 31;
    const int gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int nw = gridDim.x * (blockDim.x >> 5);
    if (k < 3) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            d[0] = A[0];
            if (k == 2) {
                e[0] = A[1];
                d[1] = A[1 + (int64_t)k];
            }
        }
        return;
    }
    // RES: owned column (A column ocol for warps 0-3, Q^T column ocol for warps 4-7) into
    // shared memory
    const int wib = threadIdx.x >> 5, ocol = blockIdx.x + gridDim.x * (wib & 3);
    const bool ownA = RES && wib < 4 && ocol < k, ownQ = RES && wib >= 4 && ocol < k;
    if (RES && (ownA || ownQ)) {
        const double *src = ownA ? A + (int64_t)ocol * k : Qt + (int64_t)ocol * k;
        for (int l = lane; l < k; l += 32) own[l] = src[l];
        __syncwarp();
    }
    // reflector 0 from column 0, and its p, q
    block_house(A, k, 1, vcur, &bcur_s, &enext_s, red);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        d[0] = A[0];
        e[0] = enext_s;
    }
    {
        const double bt = bcur_s;
        const int m = k - 1;
        for (int it = gw; it < m + k; it += nw) {
            const double *col = (it < m) ? A + (int64_t)(1 + it) * k : Qt + (int64_t)(it - m) * k;
            double s = 0.0;
            for (int l = 1 + lane; l < k; l += 32) s += col[l] * vcur[l];
            s = warp_sum(s);
            if (lane == 0) {
                if (it < m) pq[1 + it] = bt * s;           // p of column 0 in buffer 0
                else pq[2 * k + it - m] = bt * s;          // q of column 0 in buffer 0
            }
        }
    }
    grid.sync();
    for (int j = 0; j + 2 < k; ++j) {
        const int r0 = j + 1, m = k - r0, par = j & 1;
        const bool next = (j + 3 < k);   // another reflector follows (column j + 1 has rows below r0 + 1)
        const double bt = bcur_s;
        const double *p = pq + (size_t)par * k, *q = pq + 2 * (size_t)k + (size_t)par * k;
        // p and column r0 of A (rows r0..) fetched together, then K_ and w = p - K_ v
        {
            const double *a = A + (int64_t)r0 * k;
            for (int l = threadIdx.x; l < k; l += blockDim.x) {
                const bool in = (l >= r0);
                w[l] = in ? p[l] : 0.0;
                colj[l] = (in && next) ? a[l] : 0.0;
            }
        }
        // same partition of l as the fetch above (no barrier needed in between), from the
        // first l >= r0 of this thread's share: warps with no rows left issue nothing
        const int tx = threadIdx.x, nt = blockDim.x;
        const int lr = (tx >= r0) ? tx : tx + ((r0 - tx + nt - 1) / nt) * nt;
        double s = 0.0;
        for (int l = lr; l < k; l += blockDim.x) s += vcur[l] * w[l];
        const double kh = block_sum(s, red, 0.5 * bt);
        for (int l = lr; l < k; l += blockDim.x) w[l] = fma(-kh, vcur[l], w[l]);
        __syncthreads();
        double bn = 0.0;
        if (next) {
            // column r0 after this step's update, rows r0..; then reflector j + 1 from rows r0 + 1..
            const double wr = w[r0], vr = vcur[r0];
            for (int l = r0 + threadIdx.x; l < k; l += blockDim.x) colj[l] = fma(-w[l], vr, fma(-vcur[l], wr, colj[l]));
            __syncthreads();
            block_house(colj, k, r0 + 1, vnext, &bnext_s, &enext_s, red, RES);
            __syncthreads();
            if constexpr (!RES) bn = bnext_s;
            if (blockIdx.x == 0 && threadIdx.x == 0) {
                d[r0] = colj[r0];
                e[r0] = enext_s;
            }
        }
        const int r1 = r0 + 1;
        double *pn = pq + (size_t)(par ^ 1) * k, *qn = pq + 2 * (size_t)k + (size_t)(par ^ 1) * k;
        // RES: beta of the next reflector is needed only when the dot products are published
        // after the closing barrier, so a Q^T warp (the lighter update) forms its reciprocal
        // while the columns are updated, and each warp keeps its sum until then
        double tsum = 0.0;
        double *pdst = nullptr;
        if constexpr (RES) {
            if (next && threadIdx.x == 128) {
                const double den = bnext_s;
                bnext_s = (den == 0.0) ? 0.0 : rcp_fast(den);
            }
            if (ownA && ocol >= r0 && !(next && ocol == r0)) {
                const int i = ocol;
                const double vi = vcur[i], wi = w[i];
                double t = 0.0;
                for (int l = r0 + lane; l < k; l += 32) {
                    const double x = fma(-w[l], vi, fma(-vcur[l], wi, own[l]));
                    own[l] = x;
                    if (l >= r1) t = fma(x, vnext[l], t);
                }
                if (next) {
                    tsum = warp_sum(t);
                    pdst = pn + i;
                }
                // the column every CTA derives at the next step, and the last 2 x 2 block
                if (i == r1 || !next) {
                    __syncwarp();
                    double *dst = A + (int64_t)i * k;
                    for (int l = r1 - 1 + lane; l < k; l += 32) dst[l] = own[l];
                }
            } else if (ownQ) {
                const int i = ocol;
                const double qi = q[i];
                double t = 0.0;
                for (int l = r0 + lane; l < k; l += 32) {
                    const double x = own[l] - qi * vcur[l];
                    own[l] = x;
                    if (l >= r1) t = fma(x, vnext[l], t);
                }
                if (next) {
                    tsum = warp_sum(t);
                    pdst = qn + i;
                }
            }
        } else {
            for (int it = gw; it < m + k; it += nw) {
                if (it < m) {
                    const int i = r0 + it;
                    if (next && i == r0) continue;   // derived by every CTA above; never written
                    double *col = A + (int64_t)i * k;
                    const double vi = vcur[i], wi = w[i];
                    double t = 0.0;
                    for (int l0 = r0 + lane; l0 < k; l0 += 128) {   // four loads in flight per lane
                        double x[4];
#pragma unroll
                        for (int u = 0; u < 4; ++u) x[u] = (l0 + 32 * u < k) ? col[l0 + 32 * u] : 0.0;
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const int l = l0 + 32 * u;
                            if (l < k) {
                                x[u] = fma(-w[l], vi, fma(-vcur[l], wi, x[u]));
                                col[l] = x[u];
                                if (l >= r1) t = fma(x[u], vnext[l], t);
                            }
                        }
                    }
                    if (next) {
                        t = warp_sum(t);
                        if (lane == 0) pn[i] = bn * t;
                    }
                } else {
                    const int i = it - m;
                    double *col = Qt + (int64_t)i * k;
                    const double qi = q[i];
                    double t = 0.0;
                    for (int l0 = r0 + lane; l0 < k; l0 += 128) {
                        double x[4];
#pragma unroll
                        for (int u = 0; u < 4; ++u) x[u] = (l0 + 32 * u < k) ? col[l0 + 32 * u] : 0.0;
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const int l = l0 + 32 * u;
                            if (l < k) {
                                x[u] -= qi * vcur[l];
                                col[l] = x[u];
                                if (l >= r1) t = fma(x[u], vnext[l], t);
                            }
                        }
                    }
                    if (next) {
                        t = warp_sum(t);
                        if (lane == 0) qn[i] = bn * t;
                    }
                }
            }
        }
        // reflector j + 1 becomes the current one, once every warp of the CTA is done with both
        __syncthreads();
        if constexpr (RES) {
            if (next) bn = bnext_s;
            if (pdst && lane == 0) *pdst = bn * tsum;
        }
        for (int l = threadIdx.x; l < k; l += blockDim.x) vcur[l] = vnext[l];
        if (threadIdx.x == 0) bcur_s = bn;
        grid.sync();
    }
    if constexpr (RES) {
        if (ownQ) {
            double *dst = Qt + (int64_t)ocol * k;
            for (int l = lane; l < k; l += 32) dst[l] = own[l];
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        // last 2 x 2 block
        d[k - 2] = A[(k - 2) + (int64_t)(k - 2) * k];
        e[k - 2] = A[(k - 1) + (int64_t)(k - 2) * k];
        d[k - 1] = A[(k - 1) + (int64_t)(k - 1) * k];
    }
}

// Split T where |e_l| <= eps (|d_l| + |d_{l+1}|); block bounds per index; e^2;
// ||T||_inf.  One CTA of 1024 threads: split flags in parallel, block starts
// by a prefix count over 1024-index tiles, bounds written per index.
__global__ void __launch_bounds__(1024) split_kernel(const double *d, const double *e, int k, double *e2, int *blo,
                                                     int *bhi, double *tnorm, int *bstart, int *nblocks, double *ds,
                                                     double *e2s, double *tsc)
{
    __shared__ int cnt[1024];
    __shared__ double red[32];
    __shared__ int base_s, lo_carry_s;
    __shared__ double sc_s;
    const int t = threadIdx.x;
    double nrm = 0.0;
    for (int l = t; l < k; l += blockDim.x) {
        double r = fabs(d[l]);
        if (l > 0) r += fabs(e[l - 1]);
        if (l + 1 < k) r += fabs(e[l]);
        nrm = fmax(nrm, r);
    }
    for (int off = 16; off > 0; off >>= 1) nrm = fmax(nrm, __shfl_xor_sync(0xffffffffu, nrm, off));
    if ((t & 31) == 0) red[t >> 5] = nrm;
    if (t == 0) {
        base_s = 0;
        lo_carry_s = 0;
    }
    __syncthreads();
    if (t == 0) {
        double m = 0.0;
        for (int w = 0; w < 32; ++w) m = fmax(m, red[w]);
        *tnorm = m;
        // the power of two 2^-es with ||T|| 2^-es below 1: the scaled copies that the Sturm
        // counts use are exact, and their recurrences stay far from the FP64 range limits
        int es = 0;
        if (m > 0.0 && isfinite(m)) frexp(m, &es);
        sc_s = ldexp(1.0, -es);
        *tsc = sc_s;
    }
    __syncthreads();
    {
        const double sc = sc_s;
        for (int l = t; l < k; l += blockDim.x) ds[l] = d[l] * sc;
    }
    // index l ends a block when l = k - 1 or e_l is negligible
    for (int l0 = 0; l0 < k; l0 += blockDim.x) {
        const int l = l0 + t;
        bool split = false;
        if (l < k) {
            split = (l + 1 == k) || fabs(e[l]) <= DBL_EPSILON * (fabs(d[l]) + fabs(d[l + 1]));
            if (l + 1 < k) {
                e2[l] = split ? 0.0 : e[l] * e[l];
                const double es_ = split ? 0.0 : e[l] * sc_s;
                e2s[l] = es_ * es_;
            }
        }
        cnt[t] = split ? 1 : 0;
        __syncthreads();
        for (int off = 1; off < 1024; off <<= 1) {   // inclusive prefix sum
            const int v = (t >= off) ? cnt[t - off] : 0;
            __syncthreads();
            cnt[t] += v;
            __syncthreads();
        }
        const int base = base_s;
        if (l < k && split) bstart[base + cnt[t]] = l + 1;   // start of the next block
        __syncthreads();
        if (t == 0) base_s = base + cnt[1023];
        __syncthreads();
    }
    if (t == 0) {
        bstart[0] = 0;
        *nblocks = base_s;
    }
    __syncthreads();
    // bstart[b] = first index of block b, bstart[nb] = k; bounds of each index by binary search
    const int nb = base_s;
    for (int l = t; l < k; l += blockDim.x) {
        int lo = 0, hi = nb - 1;
        while (lo < hi) {   // last block b with bstart[b] <= l
            const int mid = (lo + hi + 1) >> 1;
            if (bstart[mid] <= l) lo = mid; else hi = mid - 1;
        }
        blo[l] = bstart[lo];
        bhi[l] = bstart[lo + 1] - 1;
    }
}

// Number of eigenvalues of the block [lo, hi] below x: sign changes of the
// characteristic polynomials of the leading sub-blocks, P_l = (d_l - x) P_(l-1)
// - e_(l-1)^2 P_(l-2) (Sturm), on the copies scaled by a power of two (ds, e2s, xs).
// One FMA per row on the critical path, where the ratio form q = P_l / P_(l-1)
// needs an FP64 division (a long dependent sequence on this GPU); the pair
// (P_(l-1), P_l) is rescaled by a power of two every 8 rows.  An exact zero
// counts as a sign change (a tiny negative pivot in the ratio form).
__device__ __forceinline__ long long dbits(double x) { return __double_as_longlong(x); }

__device__ __forceinline__ int sturm_count(const double *__restrict__ ds, const double *__restrict__ e2s, int lo,
                                           int hi, double xs)
{
    double p0 = 1.0, p1 = ds[lo] - xs;
    if ((dbits(p1) << 1) == 0) p1 = -DBL_MIN;
    int cnt = dbits(p1) < 0;
    int l = lo + 1;
    while (l <= hi) {
        const int lend = min(hi, l + 7);
        for (; l <= lend; ++l) {
            double p2 = fma(ds[l] - xs, p1, -e2s[l - 1] * p0);
            if ((dbits(p2) << 1) == 0) p2 = (dbits(p1) < 0) ? DBL_MIN : -DBL_MIN;
            cnt += (dbits(p2) ^ dbits(p1)) < 0;
            p0 = p1;
            p1 = p2;
        }
        // rescale by the power of two of the larger magnitude (exact)
        const int e0 = (int)((dbits(p0) >> 52) & 0x7ff), e1 = (int)((dbits(p1) >> 52) & 0x7ff);
        int sh = 1023 - max(e0, e1);
        sh = max(-1000, min(1000, sh));
        const double f = __longlong_as_double((long long)(1023 + sh) << 52);
        p0 *= f;
        p1 *= f;
    }
    return cnt;
}

// Grid point g of the pre-bracket (ascending): -||T||(1+d), -||T|| 2^(-j/8)
// (j descending), 0, +||T|| 2^(-j/8) (j descending), +||T||(1+d).
__device__ __forceinline__ double grid_point(int g, double tn)
{
    const double big = tn * (1.0 + 1e-6) + DBL_MIN;
    if (g == 0) return -big;
    if (g == kGrid - 1) return big;
    if (g == kGridHalf + 1) return 0.0;
    if (g <= kGridHalf) return -tn * exp2(-(double)(g - 1) / 8.0);
    return tn * exp2(-(double)(kGrid - 2 - g) / 8.0);
}

// counts[b * kGrid + g] = eigenvalues of block b below grid point g.
__global__ void prebracket_kernel(const double *ds, const double *e2s, const int *bstart, const int *nblocks,
                                  const double *tnorm, const double *tsc, int *counts)
{
    const int nb = *nblocks;
    const int64_t total = (int64_t)nb * kGrid;
    const double tn = *tnorm, sc = *tsc;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int b = (int)(t / kGrid), g = (int)(t - (int64_t)b * kGrid);
        const int lo = bstart[b], hi = bstart[b + 1] - 1;
        counts[t] = sturm_count(ds, e2s, lo, hi, grid_point(g, tn) * sc);
    }
}

// Multisection for one eigenvalue per segment of G lanes, U Sturm chains per
// lane: P = G U interior points per round, the bracket shrinks (P + 1)-fold.
// Fewer points per round cost more rounds but less FP64 work in total (the
// counts run on the FP64 pipe, which is narrow on this GPU).
template <int G, int U>
__global__ void multisect_kernel(const double *d, const double *ds, const double *e2s, const int *blo, const int *bhi,
                                 const int *bstart, const int *nblocks, int k, const double *tnorm, const double *tsc,
                                 const int *counts, double *w)
{
    constexpr int P = G * U;
    const int gl = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const int sl = lane % G;                                  // lane within the segment
    const unsigned seg_mask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (lane - sl));
    const int i = gl / G;
    if (i >= k) return;
    const int lo = blo[i], hi = bhi[i], r = i - lo;
    const double tn = *tnorm;
    if (lo == hi) {
        if (sl == 0) w[i] = d[lo];
        return;
    }
    // locate this block and the grid cell holding eigenvalue r
    int b = 0, nb = *nblocks, bl = 0, bh = nb - 1;
    while (bl <= bh) {
        const int mid = (bl + bh) >> 1;
        if (bstart[mid] <= lo) { b = mid; bl = mid + 1; } else bh = mid - 1;
    }
    const int *cb = counts + (int64_t)b * kGrid;
    int g0 = 0, g1 = kGrid - 1;   // cb[g0] <= r < cb[g1]
    while (g1 - g0 > 1) {
        const int gm = (g0 + g1) >> 1;
        if (cb[gm] <= r) g0 = gm; else g1 = gm;
    }
    double a = grid_point(g0, tn), c = grid_point(g1, tn);
    const double sc = *tsc;
    for (int round = 0; round < 64; ++round) {
        const double width = c - a;
        if (width <= fmax(1e-10 * fmax(fabs(a), fabs(c)), 4.0 * DBL_EPSILON * tn)) break;
        const double step = width / (double)(P + 1);
        int cnt[U];
#pragma unroll
        for (int u = 0; u < U; ++u) cnt[u] = sturm_count(ds, e2s, lo, hi, (a + step * (double)(1 + sl + G * u)) * sc);
        // the new bracket: last point with count <= r, first with count > r;
        // points ascend with (u, sl) and counts are monotone in x
        int best_le = -1, first_gt = P;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const unsigned gt = __ballot_sync(seg_mask, cnt[u] > r) >> (lane - sl);
            const unsigned le = ~gt & ((G == 32) ? 0xffffffffu : ((1u << G) - 1u));
            if (le) best_le = max(best_le, G * u + 31 - __clz(le));
            if (gt) first_gt = min(first_gt, G * u + __ffs(gt) - 1);
        }
        const double na = (best_le >= 0) ? a + step * (double)(1 + best_le) : a;
        const double nc = (first_gt < P) ? a + step * (double)(1 + first_gt) : c;
        if (!(nc - na < width)) break;   // no progress: the width is at the resolution of the arithmetic
        a = na;
        c = nc;
    }
    if (sl == 0) w[i] = 0.5 * (a + c);
}

__device__ __forceinline__ double hash_uniform(uint32_t a, uint32_t b)
{
    uint32_t h = a * 0x9E3779B1u ^ (b + 0x7F4A7C15u) * 0x85EBCA77u;
    h ^= h >> 15;
    h *= 0x2C1B3C6Du;
    h ^= h >> 12;
    h *= 0x297A2D39u;
    h ^= h >> 15;
    return ((double)h + 0.5) * 2.3283064365386963e-10 - 0.5;
}

// Inverse iteration for one eigenvalue lam of the block T_b = T[lo..lo+m-1] (dd, ee: its
// diagonal and off-diagonal), by one thread: the LU with partial pivoting of T_b - lam I,
// three solves from a pseudo-random start, normalisation and the Rayleigh quotient (written
// to *wout).  Row l of the factors sits at index l * stride of u0, u1, u2, ml and piv; z
// (unit stride, m entries) receives the eigenvector.  One FP64 reciprocal per row (of the
// pivot, kept for the back substitution; the refined hardware approximation, within one
// ulp), so the three solves are multiply-adds only; values carried from row to row stay in
// registers and the loads of the stored factors do not wait on the arithmetic.
__device__ __forceinline__ void inviter_one(uint32_t i, const double *dd, const double *ee, int m, double lam,
                                            double tiny, double *u0, double *u1, double *u2, double *ml,
                                            unsigned char *piv, int64_t stride, double *z, double *wout)
{
    if (m == 1) {
        z[0] = 1.0;
        *wout = dd[0];
        return;
    }
#define IDX(l) ((int64_t)(l) * stride)
    double a_cur = dd[0] - lam, c_cur = ee[0];
    for (int l = 0; l < m - 1; ++l) {
        const double bl = ee[l];                     // sub-diagonal below a_cur
        const double a_next = dd[l + 1] - lam;
        const double c_next = (l + 1 < m - 1) ? ee[l + 1] : 0.0;
        if (fabs(a_cur) >= fabs(bl)) {
            const double rp = rcp_fast((a_cur == 0.0) ? tiny : a_cur);
            const double mult = bl * rp;
            u0[IDX(l)] = rp;
            u1[IDX(l)] = c_cur;
            u2[IDX(l)] = 0.0;
            ml[IDX(l)] = mult;
            piv[IDX(l)] = 0;
            a_cur = a_next - mult * c_cur;
            c_cur = c_next;
        } else {
            const double rp = rcp_fast(bl);
            const double mult = a_cur * rp;
            u0[IDX(l)] = rp;
            u1[IDX(l)] = a_next;
            u2[IDX(l)] = c_next;
            ml[IDX(l)] = mult;
            piv[IDX(l)] = 1;
            a_cur = c_cur - mult * a_next;
            c_cur = -mult * c_next;
        }
    }
    u0[IDX(m - 1)] = rcp_fast((fabs(a_cur) < tiny) ? (a_cur < 0.0 ? -tiny : tiny) : a_cur);
    // start vector: distinct pseudo-random values per eigenvalue
    for (int l = 0; l < m; ++l) z[l] = hash_uniform(i, (uint32_t)l) + 1e-3;
    for (int iter = 0; iter < 3; ++iter) {
        // forward: apply the row operations (row l + 1 carried in a register); the
        // stored factors of four rows are fetched before they are used
        double carry = z[0];
        for (int l0 = 0; l0 < m - 1; l0 += 4) {
            double nx[4], mv[4];
            bool sv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int l = l0 + u;
                const bool in = l < m - 1;
                nx[u] = in ? z[l + 1] : 0.0;
                mv[u] = in ? ml[IDX(l)] : 0.0;
                sv[u] = in && piv[IDX(l)] != 0;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int l = l0 + u;
                if (l < m - 1) {
                    const double r0v = sv[u] ? nx[u] : carry, r1v = sv[u] ? carry : nx[u];
                    z[l] = r0v;
                    carry = r1v - mv[u] * r0v;
                }
            }
        }
        z[m - 1] = carry;
        // backward substitution with U (1 / diagonal, u1, u2), four rows fetched ahead
        double x2 = 0.0, x1 = 0.0, big = 0.0;
        for (int l0 = m - 1; l0 >= 0; l0 -= 4) {
            double zv[4], a0[4], a1[4], a2[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int l = l0 - u;
                const bool in = l >= 0;
                zv[u] = in ? z[l] : 0.0;
                a0[u] = in ? u0[IDX(l)] : 0.0;
                a1[u] = in ? u1[IDX(l)] : 0.0;
                a2[u] = in ? u2[IDX(l)] : 0.0;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int l = l0 - u;
                if (l >= 0) {
                    const double xl = (zv[u] - a1[u] * x1 - a2[u] * x2) * a0[u];
                    z[l] = xl;
                    x2 = x1;
                    x1 = xl;
                    big = fmax(big, fabs(xl));
                }
            }
        }
        const double sc = (big > 0.0 && isfinite(big)) ? 1.0 / big : 1.0;
        for (int l = 0; l < m; ++l) z[l] *= sc;
    }
#undef IDX
    double nrm = 0.0;
    for (int l = 0; l < m; ++l) nrm += z[l] * z[l];
    nrm = (nrm > 0.0) ? 1.0 / sqrt(nrm) : 0.0;
    for (int l = 0; l < m; ++l) z[l] *= nrm;
    // Rayleigh quotient z^T T z refines the bracketed eigenvalue
    double rq = 0.0;
    for (int l = 0; l < m; ++l) {
        double tz = dd[l] * z[l];
        if (l > 0) tz += ee[l - 1] * z[l - 1];
        if (l + 1 < m) tz += ee[l] * z[l + 1];
        rq += z[l] * tz;
    }
    *wout = rq;
}

// Inverse iteration with the factors in global memory (strided: row l of eigenvalue i at
// l * k + i) and the vector written in place, for k too large for the shared-memory form.
__global__ void inviter_kernel(const double *__restrict__ d, const double *__restrict__ e, const int *__restrict__ blo,
                               const int *__restrict__ bhi, int k, const double *__restrict__ w,
                               const double *__restrict__ tnorm, double *__restrict__ Z, double *__restrict__ u0,
                               double *__restrict__ u1, double *__restrict__ u2, double *__restrict__ ml,
                               unsigned char *__restrict__ piv, double *__restrict__ wout)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= k) return;
    const int lo = blo[i], hi = bhi[i], m = hi - lo + 1;
    double *z = Z + (int64_t)i * k;
    for (int l = 0; l < k; ++l)
        if (l < lo || l > hi) z[l] = 0.0;
    const double tiny = DBL_EPSILON * fmax(*tnorm, DBL_MIN);
    inviter_one((uint32_t)i, d + lo, e + lo, m, w[i], tiny, u0 + i, u1 + i, u2 + i, ml + i, piv + i, k, z + lo,
                wout + i);
}

// |a| >= |b| and a == 0 for finite doubles, on the integer unit: the magnitude bits of
// finite doubles order like unsigned integers (an FP64 compare would hold the FP64 unit)
__device__ __forceinline__ bool mag_ge(double a, double b)
{
    return (__double_as_longlong(a) & 0x7fffffffffffffffLL) >= (__double_as_longlong(b) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ bool is_zero(double a) { return (__double_as_longlong(a) & 0x7fffffffffffffffLL) == 0; }

// Inverse iteration for one eigenvalue by one warp, everything in shared memory (stride 1):
// lane 0 carries the serial recurrences (the LU and the two substitutions), and the passes
// that are elementwise or reductions (the scaling after each solve, the norm, the Rayleigh
// quotient) run on all 32 lanes.  One lane alone issues one FP64 instruction per ~64 cycles
// whether or not they depend on each other, so every FP64 instruction taken off lane 0's
// row loop shortens the chain.  The arithmetic is that of inviter_one, except that the
// largest entry is found after the back substitution instead of during it.
__device__ __forceinline__ void inviter_warp(uint32_t i, const double *dd, const double *ee, int m, double lam,
                                             double tiny, double *u0, double *u1, double *u2, double *ml,
                                             unsigned char *piv, double *z, double *wout, int lane)
{
    if (m == 1) {
        if (lane == 0) {
            z[0] = 1.0;
            *wout = dd[0];
        }
        return;
    }
    if (lane == 0) {
        double a_cur = dd[0] - lam, c_cur = ee[0];
        for (int l = 0; l < m - 1; ++l) {
            const double bl = ee[l];
            const double a_next = dd[l + 1] - lam;
            const double c_next = (l + 1 < m - 1) ? ee[l + 1] : 0.0;
            if (mag_ge(a_cur, bl)) {
                const double rp = rcp_fast(is_zero(a_cur) ? tiny : a_cur);
                const double mult = bl * rp;
                u0[l] = rp;
                u1[l] = c_cur;
                u2[l] = 0.0;
                ml[l] = mult;
                piv[l] = 0;
                a_cur = fma(-mult, c_cur, a_next);
                c_cur = c_next;
            } else {
                const double rp = rcp_fast(bl);
                const double mult = a_cur * rp;
                u0[l] = rp;
                u1[l] = a_next;
                u2[l] = c_next;
                ml[l] = mult;
                piv[l] = 1;
                a_cur = fma(-mult, a_next, c_cur);
                c_cur = -mult * c_next;
            }
        }
        u0[m - 1] = rcp_fast(mag_ge(a_cur, tiny) ? a_cur : (a_cur < 0.0 ? -tiny : tiny));
    }
    for (int l = lane; l < m; l += 32) z[l] = hash_uniform(i, (uint32_t)l) + 1e-3;
    __syncwarp();
    for (int iter = 0; iter < 3; ++iter) {
        if (lane == 0) {
            double carry = z[0];
            for (int l = 0; l < m - 1; ++l) {
                const double nx = z[l + 1], mv = ml[l];
                const bool sv = piv[l] != 0;
                const double r0v = sv ? nx : carry, r1v = sv ? carry : nx;
                z[l] = r0v;
                carry = fma(-mv, r0v, r1v);
            }
            z[m - 1] = carry;
            double x2 = 0.0, x1 = 0.0;
            for (int l = m - 1; l >= 0; --l) {
                const double xl = fma(-u1[l], x1, fma(-u2[l], x2, z[l])) * u0[l];
                z[l] = xl;
                x2 = x1;
                x1 = xl;
            }
        }
        __syncwarp();
        double big = 0.0;
        for (int l = lane; l < m; l += 32) big = fmax(big, fabs(z[l]));
        for (int off = 16; off > 0; off >>= 1) big = fmax(big, __shfl_xor_sync(0xffffffffu, big, off));
        const double sc = (big > 0.0 && isfinite(big)) ? 1.0 / big : 1.0;
        for (int l = lane; l < m; l += 32) z[l] *= sc;
        __syncwarp();
    }
    double nrm = 0.0;
    for (int l = lane; l < m; l += 32) nrm = fma(z[l], z[l], nrm);
    nrm = warp_sum(nrm);
    nrm = (nrm > 0.0) ? 1.0 / sqrt(nrm) : 0.0;
    double rq = 0.0;
    for (int l = lane; l < m; l += 32) {
        const double zl = z[l] * nrm;
        double tz = dd[l] * zl;
        if (l > 0) tz = fma(ee[l - 1], z[l - 1] * nrm, tz);
        if (l + 1 < m) tz = fma(ee[l], z[l + 1] * nrm, tz);
        rq = fma(zl, tz, rq);
    }
    rq = warp_sum(rq);
    __syncwarp();
    for (int l = lane; l < m; l += 32) z[l] *= nrm;
    if (lane == 0) *wout = rq;
}

// The same with T, the factors and the vector in shared memory: one warp per eigenvalue
// (inviter_warp; the pivoting branches of different eigenvalues never diverge within a
// warp, and the warp writes the column out), WPC warps per CTA sharing one copy of T.
// Shared memory: 2 k doubles of T, then per warp u0, u1, u2, ml and z (k doubles each)
// and piv (k bytes).
template <int WPC>
__global__ void __launch_bounds__(32 * WPC)
    inviter_smem_kernel(const double *__restrict__ d, const double *__restrict__ e, const int *__restrict__ blo,
                        const int *__restrict__ bhi, int k, const double *__restrict__ w,
                        const double *__restrict__ tnorm, double *__restrict__ Z, double *__restrict__ wout)
{
    extern __shared__ double ism[];
    double *ds = ism, *es = ism + k;
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double *base = ism + 2 * (size_t)k + (size_t)wib * 5 * k;
    unsigned char *pv = reinterpret_cast<unsigned char *>(ism + 2 * (size_t)k + (size_t)WPC * 5 * k) + (size_t)wib * k;
    for (int l = threadIdx.x; l < k; l += blockDim.x) {
        ds[l] = d[l];
        es[l] = (l + 1 < k) ? e[l] : 0.0;
    }
    __syncthreads();
    const int i = blockIdx.x * WPC + wib;
    if (i >= k) return;   // no CTA barrier follows
    const int lo = blo[i], hi = bhi[i], m = hi - lo + 1;
    double *zs = base + 4 * (size_t)k;
    const double tiny = DBL_EPSILON * fmax(*tnorm, DBL_MIN);
    inviter_warp((uint32_t)i, ds + lo, es + lo, m, w[i], tiny, base, base + k, base + 2 * (size_t)k,
                 base + 3 * (size_t)k, pv, zs, wout + i, lane);
    __syncwarp();
    double *z = Z + (int64_t)i * k;
    for (int l = lane; l < k; l += 32) z[l] = (l >= lo && l <= hi) ? zs[l - lo] : 0.0;
}

// Shared memory of inviter_smem_kernel<wpc> for order k.
inline size_t inviter_smem_bytes(int k, int wpc)
{
    return sizeof(double) * (2 + 5 * (size_t)wpc) * k + (size_t)wpc * k;
}

// Sort eigenvalues descending (stable by index) and gather the columns.
__global__ void eig_sort_kernel(const double *w, const double *Zt, int k, double *lam, double *Zs)
{
    const int i = blockIdx.x;
    if (i >= k) return;
    __shared__ int rank_s;
    if (threadIdx.x == 0) rank_s = 0;
    __syncthreads();
    const double wi = w[i];
    int cnt = 0;
    for (int j = threadIdx.x; j < k; j += blockDim.x) {
        const double wj = w[j];
        if (wj > wi || (wj == wi && j < i)) ++cnt;
    }
    atomicAdd(&rank_s, cnt);
    __syncthreads();
    const int rk = rank_s;
    if (threadIdx.x == 0) lam[rk] = wi;
    for (int r = threadIdx.x; r < k; r += blockDim.x) Zs[r + (int64_t)rk * k] = Zt[r + (int64_t)i * k];
}

}  // namespace

cudaError_t tridiag_eig(const double *K, int k, double *lam, double *Z, double *work, int *info, cudaStream_t s,
                        bool fp32_vectors, int *tc_err)
{
    const size_t kk = (size_t)k * k;
    double *A = work, *Qt = work + kk, *Zt = work + 2 * kk, *Zs = work + 3 * kk;
    double *u0 = work + 4 * kk, *u1 = work + 5 * kk, *u2 = work + 6 * kk, *ml = work + 7 * kk;
    unsigned char *piv = (unsigned char *)(work + 8 * kk);
    double *vec = work + 9 * kk;
    double *pq = vec, *d = vec + 4 * k, *e = vec + 5 * k;   // pq: p and q of two consecutive columns
    double *e2 = vec + 6 * k, *w = vec + 7 * k, *tnorm = vec + 8 * k + 2;
    int *blo = (int *)(vec + 9 * k), *bhi = (int *)(vec + 10 * k);
    int *bstart = (int *)(vec + 11 * k), *nblocks = (int *)(vec + 12 * k);
    double *wrq = vec + 13 * k;
    double *ds = vec + 14 * k, *e2s = vec + 15 * k, *tsc = vec + 16 * k;   // scaled copies for the Sturm counts
    int *counts = (int *)(vec + 32 * k + 1024);
    double *dinv = vec + 32 * k + 1024 + ((size_t)kGrid * k + 1) / 2 + 8;
    cudaError_t err;
    if ((err = cudaMemsetAsync(info, 0, 2 * sizeof(int), s)) != cudaSuccess) return err;
    if ((err = cudaMemsetAsync(vec, 0, sizeof(double) * 9 * k, s)) != cudaSuccess) return err;
    count_launch();
    eig_init_kernel<<<256, 256, 0, s>>>(K, k, A, Qt);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    {
        const int grid = num_sms();   // one CTA per SM keeps the grid barrier short
        // columns resident in shared memory when every column has a warp of its own
        const bool res = 2 * k <= grid * 8;
        const size_t smem = sizeof(double) * (4 * (size_t)k + kRedDoubles + (res ? 8 * (size_t)k : 0));
        const void *fn = res ? (const void *)tridiag_kernel<true> : (const void *)tridiag_kernel<false>;
        if ((err = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
            return err;
        int per_sm = 0;
        if ((err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 256, smem)) != cudaSuccess) return err;
        if (per_sm < 1) return cudaErrorInvalidConfiguration;
        void *args[] = {&A, &Qt, &k, &pq, &d, &e};
        count_launch();
        err = cudaLaunchCooperativeKernel(fn, grid, 256, args, smem, s);
        if (err != cudaSuccess) return err;
    }
    count_launch();
    split_kernel<<<1, 1024, 0, s>>>(d, e, k, e2, blo, bhi, tnorm, bstart, nblocks, ds, e2s, tsc);
    count_launch();
    prebracket_kernel<<<2 * num_sms(), 128, 0, s>>>(ds, e2s, bstart, nblocks, tnorm, tsc, counts);
    {
        // one warp of single chains per eigenvalue (33-fold shrink per round): measured on
        // k = 512 against 8 to 128 points per round, the least FP64 work that still fills the GPU
        constexpr int G = 32, U = 1;
        count_launch();
        multisect_kernel<G, U><<<(int)(((int64_t)k * G + 127) / 128), 128, 0, s>>>(d, ds, e2s, blo, bhi, bstart,
                                                                                 nblocks, k, tnorm, tsc, counts, w);
    }
    {
        // inverse iteration in shared memory when the factors of one eigenvalue fit (k <= 5670),
        // four eigenvalues per CTA where they fit (k <= 1417); else from global memory
        const size_t lim = 227 * 1024;
        count_launch();
        if (inviter_smem_bytes(k, 4) <= lim) {
            const size_t sm = inviter_smem_bytes(k, 4);
            if ((err = cudaFuncSetAttribute(inviter_smem_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)sm)) != cudaSuccess)
                return err;
            inviter_smem_kernel<4><<<(k + 3) / 4, 128, sm, s>>>(d, e, blo, bhi, k, w, tnorm, Zt, wrq);
        } else if (inviter_smem_bytes(k, 1) <= lim) {
            const size_t sm = inviter_smem_bytes(k, 1);
            if ((err = cudaFuncSetAttribute(inviter_smem_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)sm)) != cudaSuccess)
                return err;
            inviter_smem_kernel<1><<<k, 32, sm, s>>>(d, e, blo, bhi, k, w, tnorm, Zt, wrq);
        } else {
            inviter_kernel<<<(k + 3) / 4, 4, 0, s>>>(d, e, blo, bhi, k, w, tnorm, Zt, u0, u1, u2, ml, piv, wrq);
        }
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
    }
    // CholeskyQR on the eigenvectors of T: shifted passes (Fukaya et al. 2020), so that
    // eigenvalues clustered below the resolution eps ||T|| (whose inverse-iteration
    // vectors nearly coincide) still yield an orthonormal set, then a plain pass.  Two
    // shifted passes make the set orthonormal to FP64 working accuracy; one leaves it
    // within about 1e-7, enough for vectors that are used in FP32 (fp32_vectors).
    // The Grams are split over K in the LU scratch of the inverse iteration.
    const int shifted = fp32_vectors ? 1 : 2;
    if (fp32_vectors && tc_err) {
        // vectors consumed in FP32: orthonormalise their FP32 rounding as the mixed path's
        // CholeskyQR does (exact tensor-core Gram, FP64 Cholesky, one-launch FP32 solve); the
        // LU scratch holds the FP32 copy and factor, the Gram's split integers, and pq the
        // equilibration scales
        float *Zt32 = (float *)ml, *L32 = (float *)u2;
        if ((err = convert_block(Zt, 'd', k, Zt32, 'f', k, k, k, s)) != cudaSuccess) return err;
        for (int pass = 0; pass <= shifted; ++pass) {
            const double shift = pass < shifted
                                     ? fmax(11.0 * ((double)k * k + (double)k * (k + 1)) * ldexp(1.0, -53),
                                            ldexp(1.0, -29) / k)
                                     : 0.0;
            if ((err = tc_gram_f32(k, k, Zt32, k, Zs, k, u0, tc_err, s)) != cudaSuccess) return err;
            if ((err = equilibrate(Zs, k, k, Zt32, 'f', k, k, pq, s)) != cudaSuccess) return err;
            if ((err = cholesky(Zs, k, k, shift, info + (pass < shifted ? 0 : 1), dinv, s)) != cudaSuccess) return err;
            if ((err = convert_block(Zs, 'd', k, L32, 'f', k, k, k, s)) != cudaSuccess) return err;
            if ((err = put_block_inverses(L32, k, k, dinv, s)) != cudaSuccess) return err;
            if ((err = strsm_right_lt_inv(Zt32, k, k, k, L32, k, s)) != cudaSuccess) return err;
        }
        if ((err = convert_block(Zt32, 'f', k, Zt, 'd', k, k, k, s)) != cudaSuccess) return err;
    } else {
        for (int pass = 0; pass <= shifted; ++pass) {
            const double shift =
                pass < shifted ? 11.0 * ((double)k * k + (double)k * (k + 1)) * ldexp(1.0, -53) : 0.0;
            if ((err = gram_lower(k, k, Zt, 'd', k, Zs, k, s, u0, 4 * kk)) != cudaSuccess) return err;
            if ((err = cholesky(Zs, k, k, shift, info + (pass < shifted ? 0 : 1), dinv, s)) != cudaSuccess)
                return err;
            if ((err = trsm_right_lt(Zt, k, k, k, Zs, k, s, dinv)) != cudaSuccess) return err;
        }
    }
    count_launch();
    eig_sort_kernel<<<k, 128, 0, s>>>(wrq, Zt, k, lam, Zs);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    // Z = Q Zs = (Q^T)^T Zs; for vectors consumed in FP32 the product runs in FP32
    // (the LU scratch of the inverse iteration holds the FP32 copies)
    if (!fp32_vectors) return gemm('T', 'N', k, k, k, 1.0, Qt, 'd', k, Zs, 'd', k, 0.0, Z, 'd', k, s);
    float *Qt32 = (float *)u0, *Zs32 = (float *)u1, *Z32 = (float *)u2;
    if ((err = convert_block(Qt, 'd', k, Qt32, 'f', k, k, k, s)) != cudaSuccess) return err;
    if ((err = convert_block(Zs, 'd', k, Zs32, 'f', k, k, k, s)) != cudaSuccess) return err;
    if ((err = sgemm('T', 'N', k, k, k, 1.f, Qt32, k, Zs32, k, 0.f, Z32, k, s)) != cudaSuccess) return err;
    return convert_block(Z32, 'f', k, Z, 'd', k, k, k, s);
}

}  // namespace riot
