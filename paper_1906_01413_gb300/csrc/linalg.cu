// Dense linear algebra of the RIOT inner loop (column-major, FP64 arithmetic).
//
// The k x k pieces of Algorithm 3 (Gram matrices of CholeskyQR, Cholesky,
// the projected matrix K and its eigendecomposition) and the n x k x k
// products around them.  GB300 runs FP64 on the CUDA cores only, so these
// kernels are plain tiled SIMT code whose bound is the FP64 FMA rate; they
// are spread across all SMs (tile grids, row-parallel triangular solves,
// one cooperative Jacobi launch) rather than run in one CTA.
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <atomic>

#include "fp64_rcp.cuh"
#include "internal.h"

namespace cg = cooperative_groups;

namespace riot {

static std::atomic<unsigned long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
unsigned long long launches_total() { return g_launches.load(std::memory_order_relaxed); }

int num_sms()
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

// ---------------------------------------------------------------------------
// GEMM: C = alpha op(A) op(B) + beta C, double accumulation.
// 32 x 32 output tile per CTA, 256 threads, 2 x 2 outputs per thread.
// ---------------------------------------------------------------------------
template <typename TA, typename TB, typename TC>
__global__ void __launch_bounds__(256) gemm_kernel(int ta, int tb, int m, int n, int K, double alpha,
                                                   const TA *__restrict__ A, long long lda,
                                                   const TB *__restrict__ B, long long ldb, double beta,
                                                   TC *__restrict__ C, long long ldc, int lower_only, int kchunk,
                                                   long long cstride)
{
    constexpr int BM = 32, BN = 32, BK = 32;
    if (lower_only && blockIdx.y > blockIdx.x) return;   // tile strictly above the diagonal
    // split-K: z-slice z covers k in [z*kchunk, (z+1)*kchunk) and writes C + z*cstride
    const int kbeg = blockIdx.z * kchunk;
    const int kend = (kbeg + kchunk < K) ? kbeg + kchunk : K;
    C += (long long)blockIdx.z * cstride;
    __shared__ double As[BK][BM + 1];
    __shared__ double Bs[BK][BN + 1];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
    double acc[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
    for (int k0 = kbeg; k0 < kend; k0 += BK) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int idx = tid + 256 * r;
            // A tile: op(A)[i][kk], i in [m0, m0+32), kk in [k0, k0+32)
            int i, kk;
            if (!ta) { i = idx & 31; kk = idx >> 5; } else { kk = idx & 31; i = idx >> 5; }
            double va = 0.0;
            if (m0 + i < m && k0 + kk < kend)
                va = ta ? (double)A[(k0 + kk) + (long long)(m0 + i) * lda]
                        : (double)A[(m0 + i) + (long long)(k0 + kk) * lda];
            As[kk][i] = va;
            // B tile: op(B)[kk][j]
            int j;
            if (!tb) { kk = idx & 31; j = idx >> 5; } else { j = idx & 31; kk = idx >> 5; }
            double vb = 0.0;
            if (n0 + j < n && k0 + kk < kend)
                vb = tb ? (double)B[(n0 + j) + (long long)(k0 + kk) * ldb]
                        : (double)B[(k0 + kk) + (long long)(n0 + j) * ldb];
            Bs[kk][j] = vb;
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < BK; ++kk) {
            const double a0 = As[kk][tx], a1 = As[kk][tx + 16];
            const double b0 = Bs[kk][ty], b1 = Bs[kk][ty + 16];
            acc[0][0] = fma(a0, b0, acc[0][0]);
            acc[0][1] = fma(a0, b1, acc[0][1]);
            acc[1][0] = fma(a1, b0, acc[1][0]);
            acc[1][1] = fma(a1, b1, acc[1][1]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int i = m0 + tx + 16 * r, j = n0 + ty + 16 * c;
            if (i < m && j < n) {
                TC *p = C + i + (long long)j * ldc;
                const double old = (beta != 0.0) ? (double)*p : 0.0;
                *p = (TC)(alpha * acc[r][c] + beta * old);
            }
        }
}

template <typename TA, typename TB, typename TC>
static cudaError_t gemm_t(int ta, int tb, int m, int n, int k, double alpha, const void *A, int64_t lda,
                          const void *B, int64_t ldb, double beta, void *C, int64_t ldc, cudaStream_t s,
                          int lower_only = 0, int splits = 1, long long cstride = 0)
{
    if (splits < 1) splits = 1;
    int kchunk = ((k + splits - 1) / splits + 31) / 32 * 32;
    if (kchunk < 32) kchunk = 32;
    splits = (k + kchunk - 1) / kchunk;
    if (splits < 1) splits = 1;
    dim3 grid((m + 31) / 32, (n + 31) / 32, splits);
    count_launch();
    gemm_kernel<TA, TB, TC><<<grid, 256, 0, s>>>(ta, tb, m, n, k, alpha, (const TA *)A, lda, (const TB *)B, ldb,
                                                 beta, (TC *)C, ldc, lower_only, kchunk, cstride);
    return cudaGetLastError();
}

__global__ void sum_slices_lower_kernel(const double *ws, int S, int k, double *G, int64_t ldg)
{
    const int64_t total = (int64_t)k * k;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % k), j = (int)(e / k);
        if (i < j) continue;
        double s = 0.0;
        for (int z = 0; z < S; ++z) s += ws[(int64_t)z * total + e];
        G[i + (int64_t)j * ldg] = s;
    }
}

cudaError_t gram_lower(int n, int k, const void *A, char tA, int64_t lda, double *G, int64_t ldg, cudaStream_t s,
                       double *ws, size_t ws_doubles)
{
    if (k <= 0) return cudaSuccess;
    // split the long dimension when the lower tiles alone cannot fill the GPU
    const int tiles = ((k + 31) / 32) * ((k + 31) / 32 + 1) / 2;
    int S = 1;
    if (ws) {
        S = (4 * num_sms() + tiles - 1) / tiles;
        if (S > n / 128) S = n / 128;
        while (S > 1 && (size_t)S * k * k > ws_doubles) --S;
        if (S < 1) S = 1;
    }
    if (S == 1) {
        if (tA == 'd') return gemm_t<double, double, double>(1, 0, k, k, n, 1.0, A, lda, A, lda, 0.0, G, ldg, s, 1);
        if (tA == 'f') return gemm_t<float, float, double>(1, 0, k, k, n, 1.0, A, lda, A, lda, 0.0, G, ldg, s, 1);
        return cudaErrorInvalidValue;
    }
    cudaError_t e;
    const long long cs = (long long)k * k;
    if (tA == 'd') e = gemm_t<double, double, double>(1, 0, k, k, n, 1.0, A, lda, A, lda, 0.0, ws, k, s, 1, S, cs);
    else if (tA == 'f') e = gemm_t<float, float, double>(1, 0, k, k, n, 1.0, A, lda, A, lda, 0.0, ws, k, s, 1, S, cs);
    else return cudaErrorInvalidValue;
    if (e != cudaSuccess) return e;
    int kchunk = ((n + S - 1) / S + 31) / 32 * 32;
    if (kchunk < 32) kchunk = 32;
    const int Sreal = (n + kchunk - 1) / kchunk;
    count_launch();
    sum_slices_lower_kernel<<<256, 256, 0, s>>>(ws, Sreal, k, G, ldg);
    return cudaGetLastError();
}

// FP64 GEMM with 16 x 16 output tiles (one output per thread) for the thin
// updates of the blocked Cholesky and triangular solves (K = 32): FP64 issue
// per SM is the limit on this GPU, so many small tiles spread over all SMs
// finish sooner than few large ones.  lower_only skips tiles above the
// diagonal.
__global__ void __launch_bounds__(256) gemm16_kernel(int ta, int tb, int m, int n, int K, double alpha,
                                                     const double *__restrict__ A, long long lda,
                                                     const double *__restrict__ B, long long ldb, double beta,
                                                     double *__restrict__ C, long long ldc, int lower_only)
{
    if (lower_only && blockIdx.y > blockIdx.x) return;
    __shared__ double As[32][17];
    __shared__ double Bs[32][17];
    const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
    const int m0 = blockIdx.x * 16, n0 = blockIdx.y * 16;
    double acc = 0.0;
    for (int k0 = 0; k0 < K; k0 += 32) {
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int e = t + 256 * r;
            int i, kk;
            if (!ta) { i = e & 15; kk = e >> 4; } else { kk = e & 31; i = e >> 5; }
            As[kk][i] = (m0 + i < m && k0 + kk < K)
                            ? (ta ? A[(k0 + kk) + (long long)(m0 + i) * lda] : A[(m0 + i) + (long long)(k0 + kk) * lda])
                            : 0.0;
            int j;
            if (!tb) { kk = e & 31; j = e >> 5; } else { j = e & 15; kk = e >> 4; }
            Bs[kk][j] = (n0 + j < n && k0 + kk < K)
                            ? (tb ? B[(n0 + j) + (long long)(k0 + kk) * ldb] : B[(k0 + kk) + (long long)(n0 + j) * ldb])
                            : 0.0;
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < 32; ++kk) acc = fma(As[kk][tx], Bs[kk][ty], acc);
        __syncthreads();
    }
    const int i = m0 + tx, j = n0 + ty;
    if (i < m && j < n) {
        double *p = C + i + (long long)j * ldc;
        *p = alpha * acc + (beta != 0.0 ? beta * *p : 0.0);
    }
}

static cudaError_t gemm16(char ta, char tb, int m, int n, int k, double alpha, const double *A, int64_t lda,
                          const double *B, int64_t ldb, double beta, double *C, int64_t ldc, cudaStream_t s,
                          int lower_only = 0)
{
    if (m <= 0 || n <= 0) return cudaSuccess;
    dim3 grid((m + 15) / 16, (n + 15) / 16);
    count_launch();
    gemm16_kernel<<<grid, 256, 0, s>>>(ta == 'T', tb == 'T', m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, lower_only);
    return cudaGetLastError();
}

// Single-column products (y = alpha op(A) x + beta y, FP64), which the tiled
// GEMM would run at 1/32 of its lanes: y = A^T x takes one warp per output
// (lanes stride the long dimension); y = A x takes 32 rows per CTA of 8 warps,
// the warps splitting the columns, partial sums reduced in shared memory.
__global__ void __launch_bounds__(256) gemv_t_kernel(int m, int K, double alpha, const double *__restrict__ A,
                                                     long long lda, const double *__restrict__ x, double beta,
                                                     double *__restrict__ y)
{
    const int j = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (j >= m) return;
    const double *a = A + (long long)j * lda;
    double s0 = 0.0, s1 = 0.0;
    int l = lane;
    for (; l + 32 < K; l += 64) {
        s0 = fma(a[l], x[l], s0);
        s1 = fma(a[l + 32], x[l + 32], s1);
    }
    if (l < K) s0 = fma(a[l], x[l], s0);
    double v = s0 + s1;
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if (lane == 0) y[j] = alpha * v + (beta != 0.0 ? beta * y[j] : 0.0);
}

__global__ void __launch_bounds__(256) gemv_n_kernel(int m, int K, double alpha, const double *__restrict__ A,
                                                     long long lda, const double *__restrict__ x, double beta,
                                                     double *__restrict__ y)
{
    __shared__ double part[8][33];
    const int i = blockIdx.x * 32 + (threadIdx.x & 31), w = threadIdx.x >> 5;
    double v = 0.0;
    if (i < m)
        for (int l = w; l < K; l += 8) v = fma(A[i + (long long)l * lda], x[l], v);
    part[w][threadIdx.x & 31] = v;
    __syncthreads();
    if (w == 0 && i < m) {
        double t = 0.0;
#pragma unroll
        for (int r = 0; r < 8; ++r) t += part[r][threadIdx.x];
        y[i] = alpha * t + (beta != 0.0 ? beta * y[i] : 0.0);
    }
}

cudaError_t gemm(char ta, char tb, int m, int n, int k, double alpha, const void *A, char tA, int64_t lda,
                 const void *B, char tB, int64_t ldb, double beta, void *C, char tC, int64_t ldc, cudaStream_t s)
{
    if (m <= 0 || n <= 0) return cudaSuccess;
    const int a = (ta == 'T'), b = (tb == 'T');
    if (n == 1 && tb == 'N' && tA == 'd' && tB == 'd' && tC == 'd' && k > 0) {
        count_launch();
        if (a)
            gemv_t_kernel<<<(m + 7) / 8, 256, 0, s>>>(m, k, alpha, (const double *)A, lda, (const double *)B, beta,
                                                      (double *)C);
        else
            gemv_n_kernel<<<(m + 31) / 32, 256, 0, s>>>(m, k, alpha, (const double *)A, lda, (const double *)B, beta,
                                                        (double *)C);
        return cudaGetLastError();
    }
#define RIOT_GEMM_CASE(XA, XB, XC, TA_, TB_, TC_) \
    if (tA == XA && tB == XB && tC == XC) return gemm_t<TA_, TB_, TC_>(a, b, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, s);
    RIOT_GEMM_CASE('d', 'd', 'd', double, double, double)
    RIOT_GEMM_CASE('f', 'd', 'd', float, double, double)
    RIOT_GEMM_CASE('d', 'f', 'd', double, float, double)
    RIOT_GEMM_CASE('f', 'f', 'd', float, float, double)
    RIOT_GEMM_CASE('d', 'd', 'f', double, double, float)
    RIOT_GEMM_CASE('f', 'd', 'f', float, double, float)
#undef RIOT_GEMM_CASE
    return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// SGEMM (FP32 SIMT): 64 x 64 tile, BK = 16, 256 threads, 4 x 4 outputs per
// thread read as float4 from shared memory.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) sgemm_kernel(int ta, int tb, int m, int n, int K, float alpha,
                                                    const float *__restrict__ A, long long lda,
                                                    const float *__restrict__ B, long long ldb, float beta,
                                                    float *__restrict__ C, long long ldc)
{
    __shared__ __align__(16) float As[16][64];
    __shared__ __align__(16) float Bs[16][64];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int m0 = blockIdx.x * 64, n0 = blockIdx.y * 64;
    float acc[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = 0.f;
    for (int k0 = 0; k0 < K; k0 += 16) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int idx = tid + 256 * r;
            int i, kk;
            if (!ta) { i = idx & 63; kk = idx >> 6; } else { kk = idx & 15; i = idx >> 4; }
            float va = 0.f;
            if (m0 + i < m && k0 + kk < K)
                va = ta ? A[(k0 + kk) + (long long)(m0 + i) * lda] : A[(m0 + i) + (long long)(k0 + kk) * lda];
            As[kk][i] = va;
            int j;
            if (!tb) { kk = idx & 15; j = idx >> 4; } else { j = idx & 63; kk = idx >> 6; }
            float vb = 0.f;
            if (n0 + j < n && k0 + kk < K)
                vb = tb ? B[(n0 + j) + (long long)(k0 + kk) * ldb] : B[(k0 + kk) + (long long)(n0 + j) * ldb];
            Bs[kk][j] = vb;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            const float4 a4 = *reinterpret_cast<const float4 *>(&As[kk][tx * 4]);
            const float4 b4 = *reinterpret_cast<const float4 *>(&Bs[kk][ty * 4]);
            const float av[4] = {a4.x, a4.y, a4.z, a4.w}, bv[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[r][c] = fmaf(av[r], bv[c], acc[r][c]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int i = m0 + tx * 4 + r, j = n0 + ty * 4 + c;
            if (i < m && j < n) {
                float *p = C + i + (long long)j * ldc;
                *p = alpha * acc[r][c] + (beta != 0.f ? beta * *p : 0.f);
            }
        }
}

cudaError_t sgemm(char ta, char tb, int m, int n, int k, float alpha, const float *A, int64_t lda, const float *B,
                  int64_t ldb, float beta, float *C, int64_t ldc, cudaStream_t s)
{
    if (m <= 0 || n <= 0) return cudaSuccess;
    dim3 grid((m + 63) / 64, (n + 63) / 64);
    count_launch();
    sgemm_kernel<<<grid, 256, 0, s>>>(ta == 'T', tb == 'T', m, n, k, alpha, A, lda, B, ldb, beta, C, ldc);
    return cudaGetLastError();
}

// X[r, 0:jb] <- X[r, 0:jb] M^T for m rows, M the jb x jb lower-triangular
// block at Minv (ld ldm, FP32): 8 rows x 32 columns per CTA, one output per
// thread (a product with the block inverse instead of a substitution: no
// dependent chain, and enough CTAs to spread over every SM).
__global__ void __launch_bounds__(256) strmm_rows_kernel(float *X, int m, int64_t ldx, const float *Minv, int64_t ldm,
                                                         int jb)
{
    __shared__ float xs[8][33];
    __shared__ float ms[32][33];
    const int c = threadIdx.x & 31, rl = threadIdx.x >> 5;
    const int r = blockIdx.x * 8 + rl;
    for (int e = threadIdx.x; e < 32 * 32; e += blockDim.x) {
        const int i = e & 31, j = e >> 5;
        ms[i][j] = (i < jb && j < jb && j <= i) ? Minv[i + (int64_t)j * ldm] : 0.f;
    }
    xs[rl][c] = (r < m && c < jb) ? X[r + (int64_t)c * ldx] : 0.f;
    __syncthreads();
    if (r >= m || c >= jb) return;
    float acc = 0.f;
#pragma unroll 8
    for (int i = 0; i <= c; ++i) acc = fmaf(xs[rl][i], ms[c][i], acc);
    X[r + (int64_t)c * ldx] = acc;
}

// Diagonal blocks of the FP32 factor L32 (ld ldl) replaced by the FP32
// rounding of the block inverses dinv (NB x NB each, from cholesky).
__global__ void put_block_inverses_kernel(float *L32, int k, int64_t ldl, const double *dinv)
{
    const int b = blockIdx.x, J = b * 32;
    for (int e = threadIdx.x; e < 32 * 32; e += blockDim.x) {
        const int i = e & 31, j = e >> 5;
        if (J + i < k && J + j < k) L32[(J + i) + (int64_t)(J + j) * ldl] = (float)dinv[(int64_t)b * 1024 + e];
    }
}

cudaError_t put_block_inverses(float *L32, int k, int64_t ldl, const double *dinv, cudaStream_t s)
{
    if (k <= 0) return cudaSuccess;
    count_launch();
    put_block_inverses_kernel<<<(k + 31) / 32, 256, 0, s>>>(L32, k, ldl, dinv);
    return cudaGetLastError();
}

// X <- X L^-T for the rows of an m x k FP32 block in one launch (the triangular solve of a
// CholeskyQR pass; L holds the factor below its diagonal blocks and the block inverses on
// them, see put_block_inverses).  Rows are independent, so a CTA owns 32 rows for all k
// columns in shared memory (column-major over the 32 rows, four rows per float4) and sweeps
// the block columns left to right: block J takes X_J - sum_{l<J} Y_l L_Jl^T and is then
// multiplied by the block inverse.  The 32 x 32 blocks of L stream through a ring of eight
// shared-memory buffers filled by cp.async (4-byte copies, so any leading dimension works),
// seven blocks ahead of the one in use (a block's arithmetic is shorter than an L2 round
// trip).
constexpr int kTrsmRows = 32;   // rows per CTA of the tall form
constexpr int kTrsmRing = 8;

__device__ __forceinline__ void cp_async4(float *dst, const float *src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }

template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// RPT consecutive rows of one column of the row block in shared memory (a float4 for four)
template <int RPT>
__device__ __forceinline__ void ld_rows(const float *p, float *v)
{
    if constexpr (RPT == 4) {
        const float4 x = *reinterpret_cast<const float4 *>(p);
        v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
    } else {
#pragma unroll
        for (int i = 0; i < RPT; ++i) v[i] = p[i];
    }
}

template <int RPT>
__device__ __forceinline__ void st_rows(float *p, const float *v)
{
    if constexpr (RPT == 4) {
        *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
    } else {
#pragma unroll
        for (int i = 0; i < RPT; ++i) p[i] = v[i];
    }
}

// RPT rows per thread (R = 8 RPT rows per CTA): 4 for tall blocks, 1 when the rows are too few
// to give every SM a CTA of 32 (the sweep's length per CTA is the same either way, so the CTA
// with a quarter of the rows takes about a quarter of the time).
template <int RPT>
__global__ void __launch_bounds__(256) strsm_lt_rows_kernel(float *X, int m, int k, int64_t ldx, const float *L,
                                                            int64_t ldl)
{
    constexpr int R = 8 * RPT;
    extern __shared__ __align__(16) float trsm_sm[];
    float *Ys = trsm_sm;                          // [k][R]
    float *ring = trsm_sm + (size_t)k * R;        // [kTrsmRing][32 kk][32 ci]
    const int t = threadIdx.x, cj = t & 31, g = t >> 5;
    const int r0 = blockIdx.x * R;
    const int nb = (k + 31) / 32, nblk = nb * (nb + 1) / 2;
    // the rows, all in flight at once (one group, completed with the first block of L)
    for (int e = t; e < k * R; e += blockDim.x) {
        const int c = e / R, r = e - c * R;
        if (r0 + r < m) cp_async4(Ys + e, X + (r0 + r) + (int64_t)c * ldx);
        else Ys[e] = 0.f;
    }
    cp_async_commit();
    // block b of the sweep is (J, l), l = 0..J (l = J: the diagonal block)
    int iJ = 0, il = 0;   // the next block to issue
    auto issue = [&](int slot) {
        if (iJ < nb) {
            // element (ci = lane, kk = warp + 8 q) of block (iJ, il)
            float *buf = ring + slot * 1024;
            const int row = 32 * iJ + cj;
            const float *src = L + row + (int64_t)(32 * il + g) * ldl;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int kk = g + 8 * q, col = 32 * il + kk;
                if (row < k && col < k) cp_async4(buf + kk * 32 + cj, src + (int64_t)(8 * q) * ldl);
                else buf[kk * 32 + cj] = 0.f;
            }
            if (++il > iJ) {
                ++iJ;
                il = 0;
            }
        }
        cp_async_commit();
    };
#pragma unroll
    for (int q = 0; q < kTrsmRing - 1; ++q) issue(q);
    float acc[RPT];
#pragma unroll
    for (int i = 0; i < RPT; ++i) acc[i] = 0.f;
    int J = 0, l = 0;
    for (int b = 0; b < nblk; ++b) {
        cp_async_wait<kTrsmRing - 2>();
        __syncthreads();
        issue((b + kTrsmRing - 1) % kTrsmRing);
        const float *buf = ring + (b % kTrsmRing) * 1024;
        const int colJ = 32 * J + cj;
        if (l == 0) {
            if (colJ < k) {
                ld_rows<RPT>(Ys + (size_t)colJ * R + RPT * g, acc);
            } else {
#pragma unroll
                for (int i = 0; i < RPT; ++i) acc[i] = 0.f;
            }
        }
        if (l < J) {
            // eight steps of L and Y fetched before their FMAs (shared-memory latency hidden by
            // the batch rather than by other warps: one CTA of 8 warps per SM)
            const float *yb = Ys + (size_t)(32 * l) * R + RPT * g;
#pragma unroll
            for (int k0 = 0; k0 < 32; k0 += 8) {
                float a[8], y[8][RPT];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    a[u] = buf[(k0 + u) * 32 + cj];
                    ld_rows<RPT>(yb + (k0 + u) * R, y[u]);
                }
#pragma unroll
                for (int u = 0; u < 8; ++u)
#pragma unroll
                    for (int i = 0; i < RPT; ++i) acc[i] = fmaf(-y[u][i], a[u], acc[i]);
            }
            ++l;
        } else {
            // diagonal: the right-hand side through shared memory, then times the block inverse
            if (colJ < k) st_rows<RPT>(Ys + (size_t)colJ * R + RPT * g, acc);
            __syncthreads();
            const int jb = (k - 32 * J < 32) ? k - 32 * J : 32;
            float o[RPT];
#pragma unroll
            for (int i = 0; i < RPT; ++i) o[i] = 0.f;
            const float *yb = Ys + (size_t)(32 * J) * R + RPT * g;
            for (int kk = 0; kk < jb; ++kk) {
                const float a = buf[kk * 32 + cj];
                float y[RPT];
                ld_rows<RPT>(yb + kk * R, y);
#pragma unroll
                for (int i = 0; i < RPT; ++i) o[i] = fmaf(y[i], a, o[i]);
            }
            __syncthreads();
            if (colJ < k) st_rows<RPT>(Ys + (size_t)colJ * R + RPT * g, o);
            ++J;
            l = 0;
        }
    }
    cp_async_wait<0>();
    __syncthreads();
    for (int e = t; e < k * R; e += blockDim.x) {
        const int c = e / R, r = e - c * R;
        if (r0 + r < m) X[(r0 + r) + (int64_t)c * ldx] = Ys[e];
    }
}

// X <- X L^-T (X m x k FP32) where the diagonal blocks of L hold their inverses
// (put_block_inverses) and the blocks below them the factor itself: one launch of the
// row-block kernel when the rows of a block fit in shared memory, else one block column
// per launch pair.
cudaError_t strsm_right_lt_inv(float *X, int m, int k, int64_t ldx, const float *L, int64_t ldl, cudaStream_t s)
{
    if (m <= 0 || k <= 0) return cudaSuccess;
    // 32 rows per CTA while that still gives ~every SM a CTA, else 8
    const bool tall = m >= 32 * (num_sms() * 3 / 4);
    const int R = tall ? kTrsmRows : 8;
    const size_t smem = sizeof(float) * ((size_t)k * R + kTrsmRing * 1024);
    if (smem <= 227 * 1024) {
        auto kern = tall ? strsm_lt_rows_kernel<4> : strsm_lt_rows_kernel<1>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        count_launch();
        kern<<<(m + R - 1) / R, 256, smem, s>>>(X, m, k, ldx, L, ldl);
        return cudaGetLastError();
    }
    for (int J = 0; J < k; J += 32) {
        const int jb = (k - J < 32) ? k - J : 32;
        count_launch();
        strmm_rows_kernel<<<(m + 7) / 8, 256, 0, s>>>(X + (int64_t)J * ldx, m, ldx, L + J + (int64_t)J * ldl, ldl, jb);
        const int rest = k - J - jb;
        if (rest > 0) {
            cudaError_t e = sgemm('N', 'T', m, rest, jb, -1.f, X + (int64_t)J * ldx, ldx, L + (J + jb) + (int64_t)J * ldl,
                                  ldl, 1.f, X + (int64_t)(J + jb) * ldx, ldx, s);
            if (e != cudaSuccess) return e;
        }
    }
    return cudaGetLastError();
}

// C (n x n, lower triangle only) = A A^T for A n x K (FP64): the normal-equations matrix of
// the solve for K, which the Cholesky then reads from its lower triangle alone.
cudaError_t syrk_lower(int n, int K, const double *A, int64_t lda, double *C, int64_t ldc, cudaStream_t s)
{
    return gemm16('N', 'T', n, n, K, 1.0, A, lda, A, lda, 0.0, C, ldc, s, 1);
}

// ---------------------------------------------------------------------------
// Block conversion / copy
// ---------------------------------------------------------------------------
template <typename TI, typename TO>
__global__ void convert_kernel(const TI *in, int64_t ldin, TO *out, int64_t ldout, int64_t rows, int cols)
{
    const int64_t total = rows * cols;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = e / rows, i = e - j * rows;
        out[i + j * ldout] = (TO)in[i + j * ldin];
    }
}

cudaError_t convert_block(const void *in, char tin, int64_t ldin, void *out, char tout, int64_t ldout, int64_t rows,
                          int cols, cudaStream_t s)
{
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    int blocks = (int)((rows * cols + 255) / 256);
    if (blocks > 8192) blocks = 8192;
    if (tin == 'f' && tout == 'd')
        { count_launch(); convert_kernel<float, double><<<blocks, 256, 0, s>>>((const float *)in, ldin, (double *)out, ldout, rows, cols); }
    else if (tin == 'd' && tout == 'f')
        { count_launch(); convert_kernel<double, float><<<blocks, 256, 0, s>>>((const double *)in, ldin, (float *)out, ldout, rows, cols); }
    else if (tin == 'd' && tout == 'd')
        { count_launch(); convert_kernel<double, double><<<blocks, 256, 0, s>>>((const double *)in, ldin, (double *)out, ldout, rows, cols); }
    else if (tin == 'f' && tout == 'f')
        { count_launch(); convert_kernel<float, float><<<blocks, 256, 0, s>>>((const float *)in, ldin, (float *)out, ldout, rows, cols); }
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Cholesky (blocked, right-looking, nb = 32)
// ---------------------------------------------------------------------------
constexpr int NB = 32;

// G_ii += shift_scale * trace(G)  (one CTA)
__global__ void shift_diag_kernel(double *G, int k, int64_t ldg, double shift_scale)
{
    __shared__ double red[32];
    double s = 0.0;
    for (int i = threadIdx.x; i < k; i += blockDim.x) s += G[i + i * ldg];
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) t += red[w];
        red[0] = t;
    }
    __syncthreads();
    const double sh = shift_scale * red[0];
    for (int i = threadIdx.x; i < k; i += blockDim.x) G[i + i * ldg] += sh;
}

// Cholesky of the jb x jb diagonal block at (J, J) by one CTA of 256 threads (the factor
// only; the block inverses follow in one launch per factorisation).  FP64 issue costs about
// 64 cycles per warp instruction on this GPU, so the block is a chain of jb pivots: thread 0
// alone carries it while warps 1..7 apply the rank-1 update of the trailing triangle, one
// barrier per column.  The chain needs only 1 / d_j: the next pivot is
// d_(j+1) = a_(j+1,j+1) - a_(j+1,j)^2 / d_j and the updates use the unscaled columns
// (l_ij l_cj = a_ij a_cj / d_j), so each step is two FMAs and a refined hardware reciprocal
// (about 370 cycles against 560 with the library rsqrt and r * r); the square roots
// 1 / sqrt(d_j) that scale the factor are taken once, for all columns at the end.  The
// entries are enumerated from the bottom-right corner, so the trailing triangle of the last
// m columns is a prefix of the enumeration and stays spread over the update threads as it
// shrinks.  The first failing pivot is recorded in info (1-based); the factorisation
// continues with pivot 1.
__device__ __forceinline__ bool positive_finite(double d)
{
    const long long bits = __double_as_longlong(d);
    return bits > 0 && bits < 0x7ff0000000000000LL;
}

// Rank-1 update of this thread's first NQ trailing-triangle entries by column j.
template <int NQ>
__device__ __forceinline__ void potrf_update(double (*As)[NB + 1], const int *ei, const int *ec, const int *eb, int j,
                                             int m, double r2)
{
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        const int i = ei[q], c = ec[q];
        if (eb[q] < m && !(c == j + 1 && i == j + 1)) As[i][c] = fma(-As[i][j], As[c][j] * r2, As[i][c]);
    }
}

// The factorisation of a block held in shared memory (As, padded with the identity to NB x NB),
// by all 256 threads of the CTA; writes the factor to G at (J, J).  Warps 0 and 4 share a
// sub-partition (and its FP64 unit, one warp instruction per ~64 cycles): warp 0 carries the
// pivot chain and warp 4 stays idle, so no update instruction queues ahead of the chain.
__device__ void potrf_smem(double (*As)[NB + 1], double *rsq, double *rv, double *G, int64_t ldg, int J, int jb,
                           int *info)
{
    constexpr int kTri = NB * (NB - 1) / 2;   // entries of the trailing triangle after column 0
    constexpr int kUpd = 192;                 // update threads: warps 1, 2, 3, 5, 6, 7
    const int t = threadIdx.x, w = t >> 5;
    const int u = (w == 0 || w == 4) ? -1 : (w < 4 ? t - 32 : t - 64);
    // this thread's entries e = u, u + 192, u + 384: (a, b), 0 <= a <= b, b-major from the
    // corner, at row 31 - a and column 31 - b; active while b < m
    int ei[3], ec[3], eb[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const int e = u + kUpd * q;
        ei[q] = ec[q] = 0;
        eb[q] = NB;
        if (u >= 0 && e < kTri) {
            int b = (int)((sqrtf(8.f * (float)e + 1.f) - 1.f) * 0.5f);
            while ((b + 1) * (b + 2) / 2 <= e) ++b;
            while (b > 0 && b * (b + 1) / 2 > e) --b;
            const int a = e - b * (b + 1) / 2;
            ei[q] = NB - 1 - a;
            ec[q] = NB - 1 - b;
            eb[q] = b;
        }
    }
    double rcur = 0.0;   // thread 0: 1 / d_j
    if (t == 0) {
        double d = As[0][0];
        if (!positive_finite(d)) {
            atomicCAS(info, 0, J + 1);
            d = 1.0;
        }
        As[0][0] = d;
        rcur = rcp_fast(d);
        rsq[0] = rcur;
    }
    __syncthreads();
    for (int j = 0; j < NB - 1; ++j) {
        const int m = NB - 1 - j;
        if (t == 0) {
            // pivot j + 1 after this column's update (its entry is updated here only); a
            // positive finite double is a bit pattern strictly between 0 and +inf
            const double a = As[j + 1][j];
            double d = fma(-a, a * rcur, As[j + 1][j + 1]);
            if (!positive_finite(d)) {
                if (j + 1 < jb) atomicCAS(info, 0, J + j + 2);
                d = 1.0;
            }
            As[j + 1][j + 1] = d;
            rcur = rcp_fast(d);
            rsq[j + 1] = rcur;
        } else if (u >= 0) {
            // entries e >= 192 (b >= 19) are live only while j < 12 and e >= 384 (b >= 27)
            // only while j < 4: the code for them is left out after that, not predicated off,
            // since a predicated-off FP64 instruction still holds the sub-partition's unit
            const double r2 = rsq[j];
            if (j < 4)
                potrf_update<3>(As, ei, ec, eb, j, m, r2);
            else if (j < 12)
                potrf_update<2>(As, ei, ec, eb, j, m, r2);
            else
                potrf_update<1>(As, ei, ec, eb, j, m, r2);
        }
        __syncthreads();
    }
    if (t < NB) rv[t] = rsqrt(As[t][t]);   // the pivots d_c (1 on the identity padding)
    __syncthreads();
    for (int e = t; e < NB * NB; e += blockDim.x) {
        const int i = e & (NB - 1), c = e / NB;
        if (i < jb && c < jb && c <= i) G[(J + i) + (int64_t)(J + c) * ldg] = As[i][c] * rv[c];
    }
}

__global__ void __launch_bounds__(256) potrf_kernel(double *G, int64_t ldg, int J, int jb, int *info)
{
    __shared__ double As[NB][NB + 1];
    __shared__ double rsq[NB], rv[NB];
    for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
        const int i = e & (NB - 1), c = e / NB;
        As[i][c] = (i < jb && c < jb) ? (c <= i ? G[(J + i) + (int64_t)(J + c) * ldg] : 0.0) : (i == c ? 1.0 : 0.0);
    }
    __syncthreads();
    potrf_smem(As, rsq, rv, G, ldg, J, jb, info);
}

// One step of the blocked Cholesky after the panel of block column J (rows J + jb.. solved):
// the trailing update A22 -= A21 A21^T in 16 x 16 lower tiles, fused with the next diagonal
// block.  The grid runs in clusters of 2 x 2 CTAs; cluster (0, 0) (whose other three CTAs
// would be the block's own tiles or upper tiles) takes the next diagonal block: its four CTAs
// each form a quarter of the block's update from the panel rows and write it into CTA 0's
// shared memory (distributed shared memory), and after the cluster barrier CTA 0 applies it
// and factors the block at once, while the other clusters update the rest of A22.  So the
// next pivot chain starts after a quarter of the block's FP64 work instead of all of it.
__global__ void __cluster_dims__(2, 2, 1) __launch_bounds__(256)
    chol_trail_kernel(double *G, int64_t ldg, int k, int J, int jb, int *info)
{
    const int r0 = J + jb, m2 = k - r0;
    const int bx = blockIdx.x, by = blockIdx.y, t = threadIdx.x;
    __shared__ double As[NB][NB + 1];
    __shared__ double Ps[NB][NB + 1];
    __shared__ double Up[NB][NB + 1];
    __shared__ double rsq[NB], rv[NB];
    if (bx < 2 && by < 2) {
        cg::cluster_group cl = cg::this_cluster();
        const unsigned rank = cl.block_rank();
        const int jb2 = m2 < NB ? m2 : NB;
        for (int e = t; e < NB * NB; e += blockDim.x) {
            const int i = e & (NB - 1), c = e / NB;
            Ps[i][c] = (i < jb2 && c < jb) ? G[(r0 + i) + (int64_t)(J + c) * ldg] : 0.0;
            if (rank == 0)
                As[i][c] = (i < jb2 && c < jb2) ? (c <= i ? G[(r0 + i) + (int64_t)(r0 + c) * ldg] : 0.0)
                                                : (i == c ? 1.0 : 0.0);
        }
        __syncthreads();
        // lower-triangle entries e = 4 t' + rank (row-major: e -> (i, c), c <= i), 132 per CTA
        double *up0 = cl.map_shared_rank(&Up[0][0], 0);
        const int e = 4 * t + (int)rank;
        if (t < 132 && e < NB * (NB + 1) / 2) {
            int i = (int)((sqrtf(8.f * (float)e + 1.f) - 1.f) * 0.5f);
            while ((i + 1) * (i + 2) / 2 <= e) ++i;
            while (i > 0 && i * (i + 1) / 2 > e) --i;
            const int c = e - i * (i + 1) / 2;
            double a0 = 0.0, a1 = 0.0;
#pragma unroll
            for (int kk = 0; kk < NB; kk += 2) {
                a0 = fma(Ps[i][kk], Ps[c][kk], a0);
                a1 = fma(Ps[i][kk + 1], Ps[c][kk + 1], a1);
            }
            up0[i * (NB + 1) + c] = a0 + a1;
        }
        cl.sync();   // every quarter of the update is in CTA 0's shared memory
        if (rank != 0) return;
        for (int e2 = t; e2 < NB * NB; e2 += blockDim.x) {
            const int i = e2 & (NB - 1), c = e2 / NB;
            if (i < jb2 && c <= i) As[i][c] -= Up[i][c];
        }
        __syncthreads();
        potrf_smem(As, rsq, rv, G, ldg, r0, jb2, info);
        return;
    }
    if (by > bx) return;
    // tile (bx, by) of A22: rows r0 + 16 bx.., columns r0 + 16 by.. (As, Ps as [kk][16] stores)
    const int tx = t & 15, ty = t >> 4;
    const int mi = r0 + 16 * bx, nj = r0 + 16 * by;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const int e = t + 256 * q, i = e & 15, kk = e >> 4;
        As[kk][i] = (16 * bx + i < m2 && kk < jb) ? G[(mi + i) + (int64_t)(J + kk) * ldg] : 0.0;
        Ps[kk][i] = (16 * by + i < m2 && kk < jb) ? G[(nj + i) + (int64_t)(J + kk) * ldg] : 0.0;
    }
    __syncthreads();
    double a0 = 0.0, a1 = 0.0;
#pragma unroll
    for (int kk = 0; kk < NB; kk += 2) {
        a0 = fma(As[kk][tx], Ps[kk][ty], a0);
        a1 = fma(As[kk + 1][tx], Ps[kk + 1][ty], a1);
    }
    const int i = 16 * bx + tx, j = 16 * by + ty;
    if (i < m2 && j < m2 && j <= i) G[(r0 + i) + (int64_t)(r0 + j) * ldg] -= a0 + a1;
}

// A21 <- A21 L11^-T for the m2 rows below the diagonal block (L11 at L, factored): one warp
// per row, lane l holds column l.  Column c is final once the earlier columns are subtracted;
// with the columns of L11 pre-scaled by 1 / l_cc, each step is one shuffle of the unscaled
// x_c and one FMA on the later lanes (a chain of jb steps per row, all rows in parallel), and
// every lane is scaled by 1 / l_ll at the end.
__global__ void __launch_bounds__(128) panel_trsm_kernel(double *A21, int m2, int64_t lda, const double *L, int64_t ldl,
                                                         int jb)
{
    __shared__ double Ls[NB][NB + 1];   // L_lc / l_cc below the diagonal
    __shared__ double rv[NB];
    for (int i = threadIdx.x; i < NB; i += blockDim.x) rv[i] = (i < jb) ? rcp_fast(L[i + (int64_t)i * ldl]) : 0.0;
    __syncthreads();
    for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
        const int i = e & (NB - 1), c = e / NB;
        Ls[i][c] = (i < jb && c < i) ? L[i + (int64_t)c * ldl] * rv[c] : 0.0;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (r >= m2) return;
    double x = (lane < jb) ? A21[r + (int64_t)lane * lda] : 0.0;
#pragma unroll
    for (int c = 0; c < NB - 1; ++c) {
        const double xc = __shfl_sync(0xffffffffu, x, c);
        if (lane > c) x = fma(-Ls[lane][c], xc, x);
    }
    if (lane < jb) A21[r + (int64_t)lane * lda] = x * rv[lane];
}

// Inverses of all diagonal blocks of a factored lower-triangular k x k L (one CTA of 256
// threads per block, written to dinv, NB x NB column-major each).  Column c of X = L^-1 by
// right-looking substitution with lane = column: the rows are split over the 8 warps (rows
// g, g + 8, ...), so a step is one multiply by the warp that owns row i, a barrier, and at
// most four FMAs per warp on the rows below.
__device__ void trtri_block(const double *L, int k, int64_t ldl, double *dinv, int blk, double (*a)[NB + 1],
                            double (*xs)[NB + 1], double *rinv)
{
    const int J = blk * NB;
    const int jb = (k - J < NB) ? k - J : NB;
    const int t = threadIdx.x, c = t & 31, g = t >> 5;
    for (int e = t; e < NB * NB; e += blockDim.x) {
        const int i = e & (NB - 1), j = e / NB;
        a[i][j] = (i < jb && j < jb) ? L[(J + i) + (int64_t)(J + j) * ldl] : 0.0;
    }
    for (int i = t; i < NB; i += blockDim.x) rinv[i] = (i < jb) ? rcp_fast(L[(J + i) + (int64_t)(J + i) * ldl]) : 0.0;
    __syncthreads();
    double v[NB / 8];
#pragma unroll
    for (int s = 0; s < NB / 8; ++s) v[s] = (8 * s + g == c) ? 1.0 : 0.0;
#pragma unroll
    for (int i = 0; i < NB; ++i) {
        if (g == (i & 7)) {
            v[i >> 3] *= rinv[i];
            xs[i][c] = v[i >> 3];
        }
        __syncthreads();
        const double xi = xs[i][c];
        // rows 8 s + g > i; the test 8 s + 7 > i is resolved at compile time, so slots with no
        // row below i in any warp issue nothing (a predicated-off FP64 instruction still
        // holds the sub-partition's unit)
#pragma unroll
        for (int s = 0; s < NB / 8; ++s)
            if (8 * s + 7 > i && 8 * s + g > i) v[s] = fma(-a[8 * s + g][i], xi, v[s]);
    }
    double *out = dinv + (int64_t)blk * NB * NB;
#pragma unroll
    for (int s = 0; s < NB / 8; ++s) {
        const int r = 8 * s + g;
        out[r + NB * c] = (r >= c && r < jb && c < jb) ? v[s] : 0.0;
    }
}

__global__ void __launch_bounds__(256) trtri_diag_kernel(const double *L, int k, int64_t ldl, double *dinv)
{
    __shared__ double a[NB][NB + 1];
    __shared__ double xs[NB][NB + 1];   // row i of X, published when final
    __shared__ double rinv[NB];
    trtri_block(L, k, ldl, dinv, blockIdx.x, a, xs, rinv);
}

// The whole blocked Cholesky in one cooperative launch (one CTA per SM; every CTA resident,
// so grid barriers are safe), for a GPU that runs one factorisation at a time.  Per block
// column J, with L_JJ factored:
//   1. panel: every warp of the grid solves rows of A21 <- A21 L_JJ^-T (one warp per row,
//      as panel_trsm_kernel); grid barrier;
//   2. CTAs 1..8 each form a slice of the next diagonal block's update from the first rows
//      of the solved panel and count it on a flag; CTA 0 (holding the block since step 1)
//      waits for the count, subtracts, and factors the block (potrf_smem: the pivot chain),
//      while CTAs 1.. update the rest of the trailing matrix in 16 x 16 tiles (rows below the
//      next diagonal block, every column from it on); grid barrier.
// The launches of the multi-kernel form (a panel and a fused trailing step per block column)
// each paid a launch and a ramp; here a block column costs two grid barriers and one flag.
// The flag's wait is bounded (info = -1 if it ever ran out, which needs a CTA that is not
// resident, and the cooperative launch rules that out).  The block inverses come last, one
// block per CTA.
constexpr int kCoopSlices = 8;
constexpr long long kCoopPollLimit = 1LL << 22;   // a few seconds of polls (an L2 round trip and a 64 ns sleep each)

__global__ void __launch_bounds__(256, 1) chol_coop_kernel(double *G, int64_t ldg, int k, int *info, double *dinv)
{
    cg::grid_group grid = cg::this_grid();
    __shared__ double As[NB][NB + 1];
    __shared__ double Ps[NB][NB + 1];
    __shared__ double rsq[NB], rv[NB];
    const int t = threadIdx.x, lane = t & 31;
    const int nblk = (k + NB - 1) / NB;
    const int ns = (gridDim.x - 1 < kCoopSlices) ? (int)gridDim.x - 1 : kCoopSlices;   // CTAs forming the update
    unsigned *dcount = reinterpret_cast<unsigned *>(dinv + NB * (NB + 1) / 2 + 1);       // after the 528 slots
    if (blockIdx.x == 0 && t == 0) *dcount = 0u;   // visible to all after the first grid barrier
    if (blockIdx.x == 0) {
        const int jb0 = k < NB ? k : NB;
        for (int e = t; e < NB * NB; e += blockDim.x) {
            const int i = e & (NB - 1), c = e / NB;
            As[i][c] = (i < jb0 && c < jb0) ? (c <= i ? G[i + (int64_t)c * ldg] : 0.0) : (i == c ? 1.0 : 0.0);
        }
        __syncthreads();
        potrf_smem(As, rsq, rv, G, ldg, 0, jb0, info);
    }
    grid.sync();
    for (int J = 0; J + 1 < nblk; ++J) {
        const int c0 = J * NB, jb = (k - c0 < NB) ? k - c0 : NB;
        const int r0 = c0 + jb, m2 = k - r0;
        const int jb2 = m2 < NB ? m2 : NB;
        // 1. panel rows: row r to CTA r mod G, warp (r / G) mod 8, so that the rows (one
        // warp's FP64 chain each) spread over every sub-partition before any takes a second.
        // Every load a CTA needs is issued before the first use: this warp's first row, the
        // factor L_JJ, and (CTA 0) the next diagonal block, final since the previous trailing
        // update.
        const int W = gridDim.x * (blockDim.x >> 5);
        if (blockIdx.x == 0) {
#pragma unroll
            for (int q = 0; q < NB * NB / 256; ++q) {
                const int e = t + 256 * q, i = e & (NB - 1), c = e / NB;
                As[i][c] = (i < jb2 && c < jb2) ? (c <= i ? G[(r0 + i) + (int64_t)(r0 + c) * ldg] : 0.0)
                                                : (i == c ? 1.0 : 0.0);
            }
        }
        if ((int)blockIdx.x < m2) {
            const double *L = G + c0 + (int64_t)c0 * ldg;
            const int rf = blockIdx.x + gridDim.x * (t >> 5);
            const double xf = (rf < m2 && lane < jb) ? G[(r0 + rf) + (int64_t)(c0 + lane) * ldg] : 0.0;
            double lv[NB * NB / 256];
#pragma unroll
            for (int q = 0; q < NB * NB / 256; ++q) {
                const int e = t + 256 * q, i = e & (NB - 1), c = e / NB;
                lv[q] = (i < jb && c <= i) ? L[i + (int64_t)c * ldg] : 0.0;
            }
            if (t < NB) rv[t] = (t < jb) ? rcp_fast(L[t + (int64_t)t * ldg]) : 0.0;
            __syncthreads();
#pragma unroll
            for (int q = 0; q < NB * NB / 256; ++q) {
                const int e = t + 256 * q, i = e & (NB - 1), c = e / NB;
                Ps[i][c] = (c < i) ? lv[q] * rv[c] : 0.0;
            }
            __syncthreads();
            for (int r = rf; r < m2; r += W) {
                double *row = G + (r0 + r) + (int64_t)c0 * ldg;
                double x = (r == rf) ? xf : ((lane < jb) ? row[(int64_t)lane * ldg] : 0.0);
#pragma unroll
                for (int c = 0; c < NB - 1; ++c) {
                    const double xc = __shfl_sync(0xffffffffu, x, c);
                    if (lane > c) x = fma(-Ps[lane][c], xc, x);
                }
                if (lane < jb) row[(int64_t)lane * ldg] = x * rv[lane];
            }
        }
        grid.sync();
        // 2. next diagonal block (CTA 0) and the rest of the trailing update (CTAs 1..).  The
        // block's own update (528 dot products of length 32, about 4 us of FP64 issue on one
        // SM) is formed in slices by CTAs 1..ns into dinv (free until the block inverses) and
        // counted on a flag; CTA 0 waits for the count, subtracts, and runs the pivot chain.
        if (blockIdx.x == 0) {
            if (t == 0) {
                const unsigned target = (unsigned)(ns * (J + 1));
                long long polls = 0;
                while (*(volatile unsigned *)dcount < target && ++polls < kCoopPollLimit) __nanosleep(64);
                if (polls >= kCoopPollLimit) atomicCAS(info, 0, -1);   // cannot happen with every CTA resident
                __threadfence();
            }
            __syncthreads();
            for (int e = t; e < NB * (NB + 1) / 2; e += blockDim.x) {
                int i = (int)((sqrtf(8.f * (float)e + 1.f) - 1.f) * 0.5f);
                while ((i + 1) * (i + 2) / 2 <= e) ++i;
                while (i > 0 && i * (i + 1) / 2 > e) --i;
                const int c = e - i * (i + 1) / 2;
                if (i < jb2) As[i][c] -= __ldcg(dinv + e);
            }
            __syncthreads();
            potrf_smem(As, rsq, rv, G, ldg, r0, jb2, info);
        } else {
            if (blockIdx.x <= ns) {
                // slice blockIdx.x - 1: entries [e0, e0 + per), one thread per entry, in the
                // summation order of chol_trail_kernel (so both forms give the same factor)
                const int per = (NB * (NB + 1) / 2 + ns - 1) / ns, e0 = (blockIdx.x - 1) * per;
#pragma unroll
                for (int q = 0; q < NB * NB / 256; ++q) {
                    const int e = t + 256 * q, i = e & (NB - 1), c = e / NB;
                    Ps[i][c] = (i < jb2 && c < jb) ? G[(r0 + i) + (int64_t)(c0 + c) * ldg] : 0.0;
                }
                __syncthreads();
                const int e = e0 + t;
                if (t < per && e < NB * (NB + 1) / 2) {
                    int i = (int)((sqrtf(8.f * (float)e + 1.f) - 1.f) * 0.5f);
                    while ((i + 1) * (i + 2) / 2 <= e) ++i;
                    while (i > 0 && i * (i + 1) / 2 > e) --i;
                    const int c = e - i * (i + 1) / 2;
                    double a0 = 0.0, a1 = 0.0;
#pragma unroll
                    for (int kk = 0; kk < NB; kk += 2) {
                        a0 = fma(Ps[i][kk], Ps[c][kk], a0);
                        a1 = fma(Ps[i][kk + 1], Ps[c][kk + 1], a1);
                    }
                    dinv[e] = a0 + a1;
                }
                __threadfence();
                __syncthreads();
                if (t == 0) atomicAdd(dcount, 1u);
            }
            // tiles: rows r0 + jb2 + 16 tr.. (m3 rows), columns r0 + 16 tc.. (m2 columns); a
            // tile holds a lower entry only if tc <= tr + 2
            const int m3 = m2 - jb2, nr = (m3 + 15) / 16, nc = (m2 + 15) / 16;
            const int tx = t & 15, ty = t >> 4;
            for (int tt = blockIdx.x - 1; tt < nr * nc; tt += gridDim.x - 1) {
                const int tr = tt / nc, tc = tt - tr * nc;
                if (tc > tr + 2) continue;   // uniform over the CTA
                const int mi = r0 + jb2 + 16 * tr, nj = r0 + 16 * tc;
                __syncthreads();   // the previous tile's reads of As / Ps are done
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const int e = t + 256 * q, i = e & 15, kk = e >> 4;
                    As[kk][i] = (mi + i < k && kk < jb) ? G[(mi + i) + (int64_t)(c0 + kk) * ldg] : 0.0;
                    Ps[kk][i] = (nj + i < k && kk < jb) ? G[(nj + i) + (int64_t)(c0 + kk) * ldg] : 0.0;
                }
                __syncthreads();
                const int i = mi + tx, j = nj + ty;
                if (i < k && j <= i) {
                    double a0 = 0.0, a1 = 0.0;
#pragma unroll
                    for (int kk = 0; kk < NB; kk += 2) {
                        a0 = fma(As[kk][tx], Ps[kk][ty], a0);
                        a1 = fma(As[kk + 1][tx], Ps[kk + 1][ty], a1);
                    }
                    G[i + (int64_t)j * ldg] -= a0 + a1;
                }
            }
        }
        grid.sync();
    }
    // block inverses, one block per CTA (As, Ps, rv as the work arrays)
    for (int b = blockIdx.x; b < nblk; b += gridDim.x) {
        __syncthreads();
        trtri_block(G, k, ldg, dinv, b, As, Ps, rv);
    }
}

// X[r, 0:jb] <- X[r, 0:jb] M^T (trans = 1) or X[r, 0:jb] M (trans = 0) in
// place for m rows, M = the jb x jb lower-triangular block at Minv (ld NB).
// 8 rows x 32 columns per CTA: each thread forms one output entry.
__global__ void __launch_bounds__(256) trmm_rows_kernel(double *X, int m, int64_t ldx, const double *Minv, int jb,
                                                        int trans)
{
    __shared__ double xs[8][NB + 1];
    __shared__ double ms[NB][NB + 1];
    const int c = threadIdx.x & 31, rl = threadIdx.x >> 5;
    const int r = blockIdx.x * 8 + rl;
    for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) ms[e % NB][e / NB] = Minv[e];
    xs[rl][c] = (r < m && c < jb) ? X[r + (int64_t)c * ldx] : 0.0;
    __syncthreads();
    if (r >= m || c >= jb) return;
    double acc = 0.0;
    if (trans) {
        // (X M^T)_c = sum_{i <= c} x_i M[c][i]
#pragma unroll 8
        for (int i = 0; i <= c; ++i) acc = fma(xs[rl][i], ms[c][i], acc);
    } else {
        // (X M)_c = sum_{i >= c} x_i M[i][c]
#pragma unroll 8
        for (int i = c; i < jb; ++i) acc = fma(xs[rl][i], ms[i][c], acc);
    }
    X[r + (int64_t)c * ldx] = acc;
}

// X[r, 0:jb] <- X[r, 0:jb] L^-T for each row r (L = the jb x jb lower block
// at Ld with leading dimension ldl).  Right-looking: once x_j is known it is
// subtracted from all later entries, so each step is one multiply plus
// independent FMAs (short dependency chains for the long FP64 latency).
__global__ void trsm_rows_lt_kernel(double *X, int m, int64_t ldx, const double *Ld, int64_t ldl, int jb)
{
    __shared__ double Ls[NB][NB + 1];
    __shared__ double rinv[NB];
    for (int e = threadIdx.x; e < jb * jb; e += blockDim.x) {
        const int i = e % jb, j = e / jb;
        Ls[i][j] = Ld[i + (int64_t)j * ldl];
    }
    for (int j = threadIdx.x; j < jb; j += blockDim.x) rinv[j] = 1.0 / Ld[j + (int64_t)j * ldl];
    __syncthreads();
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= m) return;
    double x[NB];
#pragma unroll
    for (int j = 0; j < NB; ++j) x[j] = (j < jb) ? X[r + (int64_t)j * ldx] : 0.0;
#pragma unroll
    for (int j = 0; j < NB; ++j) {
        if (j < jb) {
            x[j] *= rinv[j];
#pragma unroll
            for (int i = j + 1; i < NB; ++i)
                if (i < jb) x[i] = fma(-x[j], Ls[i][j], x[i]);
        }
    }
#pragma unroll
    for (int j = 0; j < NB; ++j)
        if (j < jb) X[r + (int64_t)j * ldx] = x[j];
}

// X[r, 0:jb] <- X[r, 0:jb] L^-1 (L lower): right-looking from the last column.
__global__ void trsm_rows_l_kernel(double *X, int m, int64_t ldx, const double *Ld, int64_t ldl, int jb)
{
    __shared__ double Ls[NB][NB + 1];
    __shared__ double rinv[NB];
    for (int e = threadIdx.x; e < jb * jb; e += blockDim.x) {
        const int i = e % jb, j = e / jb;
        Ls[i][j] = Ld[i + (int64_t)j * ldl];
    }
    for (int j = threadIdx.x; j < jb; j += blockDim.x) rinv[j] = 1.0 / Ld[j + (int64_t)j * ldl];
    __syncthreads();
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= m) return;
    double x[NB];
#pragma unroll
    for (int j = 0; j < NB; ++j) x[j] = (j < jb) ? X[r + (int64_t)j * ldx] : 0.0;
#pragma unroll
    for (int jj = NB - 1; jj >= 0; --jj) {
        if (jj < jb) {
            x[jj] *= rinv[jj];
#pragma unroll
            for (int i = 0; i < jj; ++i) x[i] = fma(-x[jj], Ls[jj][i], x[i]);
        }
    }
#pragma unroll
    for (int j = 0; j < NB; ++j)
        if (j < jb) X[r + (int64_t)j * ldx] = x[j];
}

size_t dinv_doubles(int k) { return (size_t)((k + NB - 1) / NB) * NB * NB; }

cudaError_t cholesky(double *G, int k, int64_t ldg, double shift_scale, int *info, double *dinv, cudaStream_t s,
                     bool whole_gpu)
{
    cudaError_t e = cudaMemsetAsync(info, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    if (shift_scale > 0.0) { count_launch(); shift_diag_kernel<<<1, 1024, 0, s>>>(G, k, ldg, shift_scale); }
    if (whole_gpu && k > NB) {
        void *args[] = {(void *)&G, (void *)&ldg, (void *)&k, (void *)&info, (void *)&dinv};
        count_launch();
        e = cudaLaunchCooperativeKernel((const void *)chol_coop_kernel, num_sms(), 256, args, 0, s);
        return e;
    }
    // potrf of block 0, then per block column: the panel below it, and the trailing update
    // fused with the factorisation of the next diagonal block
    { count_launch(); potrf_kernel<<<1, 256, 0, s>>>(G, ldg, 0, k < NB ? k : NB, info); }
    for (int J = 0; J < k; J += NB) {
        const int jb = (k - J < NB) ? k - J : NB;
        const int m2 = k - J - jb;
        if (m2 <= 0) break;
        double *A21 = G + (J + jb) + (int64_t)J * ldg;
        { count_launch(); panel_trsm_kernel<<<(m2 + 3) / 4, 128, 0, s>>>(A21, m2, ldg, G + J + (int64_t)J * ldg, ldg, jb); }
        const int nt = ((m2 + 15) / 16 + 1) & ~1;   // clusters of 2 x 2 CTAs
        { count_launch(); chol_trail_kernel<<<dim3(nt, nt), 256, 0, s>>>(G, ldg, k, J, jb, info); }
    }
    // the block inverses that the triangular solves multiply by
    count_launch();
    trtri_diag_kernel<<<(k + NB - 1) / NB, 256, 0, s>>>(G, k, ldg, dinv);
    return cudaGetLastError();
}

cudaError_t trtri_diag(const double *L, int k, int64_t ldl, double *dinv, cudaStream_t s)
{
    count_launch();
    trtri_diag_kernel<<<(k + NB - 1) / NB, 256, 0, s>>>(L, k, ldl, dinv);
    return cudaGetLastError();
}

// X <- X L^-T (LT) or X L^-1 in one launch, FP64: rows are independent, so a CTA of four
// warps owns four rows (one per warp: a sub-partition each, since FP64 throughput per
// sub-partition bounds this kernel) for all k columns in shared memory and sweeps the block
// columns (forward for L^-T, backward for L^-1): block J takes X_J minus the finished blocks
// times the matching blocks of L, then the block inverse from cholesky.  The 32 x 32 blocks of
// L go through a shared buffer (coalesced copy, then read along either index), the next one
// fetched into registers while the current one is used.
template <bool LT>
__global__ void __launch_bounds__(128) dtrsm_rows_kernel(double *X, int m, int k, int64_t ldx, const double *L,
                                                         int64_t ldl, const double *dinv)
{
    extern __shared__ double dtrsm_sm[];
    double *ys = dtrsm_sm;                                                                   // [4][k]
    double (*Ls)[NB + 1] = reinterpret_cast<double (*)[NB + 1]>(dtrsm_sm + 4 * (size_t)k);   // [2 NB][NB + 1]
    const int t = threadIdx.x, r = t >> 5, c = t & 31;
    const int r0 = blockIdx.x * 4;
    const int nb = (k + NB - 1) / NB;
    for (int e = t; e < 4 * k; e += blockDim.x) {
        const int cc = e >> 2, rr = e & 3;
        ys[rr * k + cc] = (r0 + rr < m) ? X[(r0 + rr) + (int64_t)cc * ldx] : 0.0;
    }
    // targets T in sweep order; target T's source blocks q = 0 .. nsrc(T) - 1 are L_{T,q}
    // (L^-T: q < T) or L_{nb-1-q, T} (L^-1); the next source block to fetch is (fT, fq)
    auto nsrc = [&](int T) { return LT ? T : nb - 1 - T; };
    auto src_block = [&](int T, int q, int &bi, int &bj) {
        if (LT) { bi = T; bj = q; }
        else { bi = nb - 1 - q; bj = T; }
    };
    int fT = LT ? 1 : nb - 2, fq = 0;
    auto has_next = [&]() { return LT ? fT < nb : fT >= 0; };
    auto advance = [&]() {
        if (++fq == nsrc(fT)) {
            fT += LT ? 1 : -1;
            fq = 0;
        }
    };
    double pre[8];
    auto fetch = [&]() {
        int bi, bj;
        src_block(fT, fq, bi, bj);
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int e = t + 128 * u, i = e & 31, j = e >> 5;
            const int gi = NB * bi + i, gj = NB * bj + j;
            pre[u] = (gi < k && gj < k) ? L[gi + (int64_t)gj * ldl] : 0.0;
        }
        advance();
    };
    if (has_next()) fetch();
    __syncthreads();
    int buf = 0;
    for (int jj = 0; jj < nb; ++jj) {
        const int T = LT ? jj : nb - 1 - jj;
        const int colT = NB * T + c;
        double acc0 = (colT < k) ? ys[r * k + colT] : 0.0, acc1 = 0.0;
        for (int q = 0; q < nsrc(T); ++q) {
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int e = t + 128 * u;
                Ls[buf * NB + (e & 31)][e >> 5] = pre[u];
            }
            __syncthreads();
            if (has_next()) fetch();
            int bi, bj;
            src_block(T, q, bi, bj);
            const double(*B)[NB + 1] = Ls + buf * NB;
            const double *yb = ys + r * k + NB * (LT ? bj : bi);
#pragma unroll 8
            for (int kk = 0; kk < NB; kk += 2) {
                const double b0 = LT ? B[c][kk] : B[kk][c], b1 = LT ? B[c][kk + 1] : B[kk + 1][c];
                acc0 = fma(-yb[kk], b0, acc0);
                acc1 = fma(-yb[kk + 1], b1, acc1);
            }
            buf ^= 1;
        }
        // diagonal: the right-hand side through shared memory, then times the block inverse
        const double *D = dinv + (int64_t)T * NB * NB;   // column-major, lower
        const int jb = (k - NB * T < NB) ? k - NB * T : NB;
        __syncthreads();
        if (colT < k) ys[r * k + colT] = acc0 + acc1;
        __syncthreads();
        double o = 0.0;
        for (int kk = 0; kk < jb; ++kk) o = fma(ys[r * k + NB * T + kk], LT ? D[c + NB * kk] : D[kk + NB * c], o);
        __syncthreads();
        if (colT < k) ys[r * k + colT] = o;
    }
    __syncthreads();
    for (int e = t; e < 4 * k; e += blockDim.x) {
        const int cc = e >> 2, rr = e & 3;
        if (r0 + rr < m) X[(r0 + rr) + (int64_t)cc * ldx] = ys[rr * k + cc];
    }
}

static cudaError_t dtrsm_rows(double *X, int m, int k, int64_t ldx, const double *L, int64_t ldl, const double *dinv,
                              bool lt, cudaStream_t s)
{
    const size_t smem = sizeof(double) * (4 * (size_t)k + 2 * NB * (NB + 1));
    auto kern = lt ? dtrsm_rows_kernel<true> : dtrsm_rows_kernel<false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    count_launch();
    kern<<<(m + 3) / 4, 128, smem, s>>>(X, m, k, ldx, L, ldl, dinv);
    return cudaGetLastError();
}

cudaError_t trsm_right_lt(double *X, int m, int k, int64_t ldx, const double *L, int64_t ldl, cudaStream_t s,
                          const double *dinv)
{
    if (m <= 0 || k <= 0) return cudaSuccess;
    if (sizeof(double) * (4 * (size_t)k + 2 * NB * (NB + 1)) <= 227 * 1024) return dtrsm_rows(X, m, k, ldx, L, ldl, dinv, true, s);
    for (int J = 0; J < k; J += NB) {
        const int jb = (k - J < NB) ? k - J : NB;
        count_launch();
        trmm_rows_kernel<<<(m + 7) / 8, 256, 0, s>>>(X + (int64_t)J * ldx, m, ldx, dinv + (int64_t)(J / NB) * NB * NB,
                                                     jb, 1);
        const int rest = k - J - jb;
        if (rest > 0) {
            cudaError_t e = gemm16('N', 'T', m, rest, jb, -1.0, X + (int64_t)J * ldx, ldx, L + (J + jb) + (int64_t)J * ldl,
                                   ldl, 1.0, X + (int64_t)(J + jb) * ldx, ldx, s);
            if (e != cudaSuccess) return e;
        }
    }
    return cudaGetLastError();
}

cudaError_t trsm_right_l(double *X, int m, int k, int64_t ldx, const double *L, int64_t ldl, cudaStream_t s,
                         const double *dinv)
{
    if (m <= 0 || k <= 0) return cudaSuccess;
    if (sizeof(double) * (4 * (size_t)k + 2 * NB * (NB + 1)) <= 227 * 1024) return dtrsm_rows(X, m, k, ldx, L, ldl, dinv, false, s);
    const int nblk = (k + NB - 1) / NB;
    for (int b = nblk - 1; b >= 0; --b) {
        const int J = b * NB;
        const int jb = (k - J < NB) ? k - J : NB;
        count_launch();
        trmm_rows_kernel<<<(m + 7) / 8, 256, 0, s>>>(X + (int64_t)J * ldx, m, ldx, dinv + (int64_t)b * NB * NB, jb, 0);
        if (J > 0) {
            cudaError_t e = gemm16('N', 'N', m, J, jb, -1.0, X + (int64_t)J * ldx, ldx, L + J, ldl, 1.0, X, ldx, s);
            if (e != cudaSuccess) return e;
        }
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Symmetric eigendecomposition: parallel cyclic Jacobi (round-robin pairs).
// Each round applies ke/2 disjoint rotations at once: A <- J^T A J on 2 x 2
// blocks (double-buffered), V <- V J.  A sweep is ke-1 rounds; iteration
// stops after a sweep in which no pair needed a rotation, i.e.
// |a_pq| <= tol * sqrt(|a_pp a_qq|) everywhere (relative-accuracy
// threshold of Demmel & Veselic).
// ---------------------------------------------------------------------------
size_t jacobi_work_doubles(int k)
{
    const size_t ke = (size_t)(k + (k & 1));
    return 3 * ke * ke + 256 + ke;
}

__device__ __forceinline__ int rr_player(int x, int r, int ke)
{
    return x == 0 ? 0 : ((x - 1 + r) % (ke - 1)) + 1;
}

__device__ __forceinline__ void jac_rot(double app, double aqq, double apq, double tol, double floor_abs, double &c,
                                        double &s, bool &rot)
{
    if (fabs(apq) <= tol * sqrt(fabs(app * aqq)) || fabs(apq) <= floor_abs) {
        c = 1.0; s = 0.0; rot = false;
        return;
    }
    const double tau = (aqq - app) / (2.0 * apq);
    const double t = (tau >= 0.0) ? 1.0 / (tau + sqrt(1.0 + tau * tau)) : -1.0 / (-tau + sqrt(1.0 + tau * tau));
    c = 1.0 / sqrt(1.0 + t * t);
    s = t * c;
    rot = true;
}

__global__ void jacobi_init_kernel(const double *K, int k, int ke, double *A0, double *V)
{
    const int64_t total = (int64_t)ke * ke;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % ke), j = (int)(e / ke);
        A0[e] = (i < k && j < k) ? 0.5 * (K[i + (int64_t)j * k] + K[j + (int64_t)i * k]) : 0.0;
        V[e] = (i == j) ? 1.0 : 0.0;
    }
}

__global__ void __launch_bounds__(256) jacobi_kernel(double *Abuf, double *V, int ke, double tol, int maxsweeps,
                                                     int *counters, int *info, double *rot)
{
    cg::grid_group grid = cg::this_grid();
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    const int64_t gtid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int half = ke / 2;
    double *Ain = Abuf, *Aout = Abuf + (int64_t)ke * ke;
    double *rc = rot, *rs = rot + half;
    // ||A||_F^2 for the absolute rotation floor (rounding level of the input)
    double *frob = (double *)(counters + 128);
    double part = 0.0;
    for (int64_t e = gtid; e < (int64_t)ke * ke; e += nthreads) part += Ain[e] * Ain[e];
    for (int off = 16; off > 0; off >>= 1) part += __shfl_down_sync(0xffffffffu, part, off);
    if ((threadIdx.x & 31) == 0 && part != 0.0) atomicAdd(frob, part);
    grid.sync();
    const double floor_abs = 1e-17 * sqrt(*((volatile double *)frob));
    int sweep = 0;
    for (; sweep < maxsweeps; ++sweep) {
        int myrot = 0;
        for (int r = 0; r < ke - 1; ++r) {
            // rotation of every pair of this round, once
            for (int64_t P = gtid; P < half; P += nthreads) {
                int p = rr_player((int)P, r, ke), q = rr_player(ke - 1 - (int)P, r, ke);
                if (p > q) { int tmp = p; p = q; q = tmp; }
                double c, sn;
                bool rt;
                jac_rot(Ain[p + (int64_t)p * ke], Ain[q + (int64_t)q * ke], Ain[p + (int64_t)q * ke], tol, floor_abs, c,
                        sn, rt);
                rc[P] = c;
                rs[P] = rt ? sn : 0.0;
                if (rt) ++myrot;
            }
            grid.sync();
            // A <- J^T A J on all 2 x 2 blocks
            for (int64_t e = gtid; e < (int64_t)half * half; e += nthreads) {
                const int P = (int)(e % half), Q = (int)(e / half);
                int p = rr_player(P, r, ke), q = rr_player(ke - 1 - P, r, ke);
                if (p > q) { int tmp = p; p = q; q = tmp; }
                int u = rr_player(Q, r, ke), w = rr_player(ke - 1 - Q, r, ke);
                if (u > w) { int tmp = u; u = w; w = tmp; }
                const double cP = rc[P], sP = rs[P], cQ = rc[Q], sQ = rs[Q];
                const double apu = Ain[p + (int64_t)u * ke], apw = Ain[p + (int64_t)w * ke];
                const double aqu = Ain[q + (int64_t)u * ke], aqw = Ain[q + (int64_t)w * ke];
                // T = blk R_Q
                const double t00 = apu * cQ - apw * sQ, t01 = apu * sQ + apw * cQ;
                const double t10 = aqu * cQ - aqw * sQ, t11 = aqu * sQ + aqw * cQ;
                // R_P^T T
                double n00 = cP * t00 - sP * t10, n01 = cP * t01 - sP * t11;
                double n10 = sP * t00 + cP * t10, n11 = sP * t01 + cP * t11;
                if (P == Q && sP != 0.0) { n01 = 0.0; n10 = 0.0; }
                Aout[p + (int64_t)u * ke] = n00;
                Aout[p + (int64_t)w * ke] = n01;
                Aout[q + (int64_t)u * ke] = n10;
                Aout[q + (int64_t)w * ke] = n11;
            }
            // V <- V J
            for (int64_t e = gtid; e < (int64_t)ke * half; e += nthreads) {
                const int i = (int)(e % ke), P = (int)(e / ke);
                const double s_ = rs[P];
                if (s_ != 0.0) {
                    int p = rr_player(P, r, ke), q = rr_player(ke - 1 - P, r, ke);
                    if (p > q) { int tmp = p; p = q; q = tmp; }
                    const double c = rc[P];
                    const double vp = V[i + (int64_t)p * ke], vq = V[i + (int64_t)q * ke];
                    V[i + (int64_t)p * ke] = vp * c - vq * s_;
                    V[i + (int64_t)q * ke] = vp * s_ + vq * c;
                }
            }
            grid.sync();
            double *tmp = Ain; Ain = Aout; Aout = tmp;
        }
        if (myrot) atomicAdd(&counters[sweep], myrot);
        grid.sync();
        const int nrot = *((volatile int *)&counters[sweep]);
        if (nrot == 0) break;
    }
    if (gtid == 0) {
        info[0] = (sweep < maxsweeps) ? sweep + 1 : -maxsweeps;
        info[1] = (Ain == Abuf) ? 0 : 1;   // which buffer holds the result
    }
}

// Sort eigenvalues descending (stable by index), gather eigenvectors with sign fix.
__global__ void jacobi_finish_kernel(const double *Abuf, const double *V, const int *info, int k, int ke, double *lam,
                                     double *Z)
{
    const double *A = Abuf + (info[1] ? (int64_t)ke * ke : 0);
    const int i = blockIdx.x;  // one CTA per eigenpair (source index i)
    if (i >= k) return;
    const double li = A[i + (int64_t)i * ke];
    __shared__ int rank_s;
    __shared__ double best_s[32];
    __shared__ int bidx_s[32];
    if (threadIdx.x == 0) rank_s = 0;
    __syncthreads();
    int cnt = 0;
    for (int j = threadIdx.x; j < k; j += blockDim.x) {
        const double lj = A[j + (int64_t)j * ke];
        if (lj > li || (lj == li && j < i)) ++cnt;
    }
    atomicAdd(&rank_s, cnt);
    // sign: largest-magnitude component positive (first one on ties)
    double best = -1.0;
    int bidx = 0;
    for (int r = threadIdx.x; r < k; r += blockDim.x) {
        const double v = fabs(V[r + (int64_t)i * ke]);
        if (v > best) { best = v; bidx = r; }
    }
    for (int off = 16; off > 0; off >>= 1) {
        const double ob = __shfl_down_sync(0xffffffffu, best, off);
        const int oi = __shfl_down_sync(0xffffffffu, bidx, off);
        if (ob > best || (ob == best && oi < bidx)) { best = ob; bidx = oi; }
    }
    if ((threadIdx.x & 31) == 0) { best_s[threadIdx.x >> 5] = best; bidx_s[threadIdx.x >> 5] = bidx; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x + 31) / 32; ++w)
            if (best_s[w] > best_s[0] || (best_s[w] == best_s[0] && bidx_s[w] < bidx_s[0])) {
                best_s[0] = best_s[w];
                bidx_s[0] = bidx_s[w];
            }
    }
    __syncthreads();
    const double sgn = (V[bidx_s[0] + (int64_t)i * ke] < 0.0) ? -1.0 : 1.0;
    const int rk = rank_s;
    if (threadIdx.x == 0) lam[rk] = li;
    for (int r = threadIdx.x; r < k; r += blockDim.x) Z[r + (int64_t)rk * k] = sgn * V[r + (int64_t)i * ke];
}

cudaError_t jacobi_eig(double *K, int k, double *lam, double *Z, double *work, int *info, cudaStream_t s)
{
    const int ke = k + (k & 1);
    double *Abuf = work;                         // 2 ke^2
    double *V = work + 2 * (size_t)ke * ke;       // ke^2
    int *counters = (int *)(V + (size_t)ke * ke); // 128 ints, then the Frobenius accumulator
    double *rot = V + (size_t)ke * ke + 256;       // cos / sin of the ke/2 pairs of a round
    const int maxsweeps = 60;
    cudaError_t e = cudaMemsetAsync(counters, 0, 128 * sizeof(int) + 2 * sizeof(double), s);
    if (e != cudaSuccess) return e;
    { count_launch(); jacobi_init_kernel<<<256, 256, 0, s>>>(K, k, ke, Abuf, V); }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (ke >= 2) {
        int dev = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, jacobi_kernel, 256, 0);
        if (per_sm < 1) per_sm = 1;
        int need = (int)(((int64_t)(ke / 2) * (ke / 2) + 255) / 256);
        int grid = num_sms() * per_sm;
        if (grid > need) grid = need;
        if (grid < 1) grid = 1;
        double tol = 1e-15 * (double)(k > 16 ? k : 16) * 0.0625;
        void *args[] = {&Abuf, &V, (void *)&ke, &tol, (void *)&maxsweeps, &counters, &info, &rot};
        count_launch();
        e = cudaLaunchCooperativeKernel((void *)jacobi_kernel, grid, 256, args, 0, s);
        if (e != cudaSuccess) return e;
    } else {
        int one[2] = {1, 0};
        e = cudaMemcpyAsync(info, one, sizeof(one), cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return e;
    }
    { count_launch(); jacobi_finish_kernel<<<k, 128, 0, s>>>(Abuf, V, info, k, ke, lam, Z); }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Small elementwise helpers
// ---------------------------------------------------------------------------
__global__ void symmetrize_kernel(double *A, int k, int64_t lda)
{
    const int64_t total = (int64_t)k * k;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % k), j = (int)(e / k);
        if (i < j) {
            const double v = 0.5 * (A[i + j * lda] + A[j + i * lda]);
            A[i + j * lda] = v;
            A[j + i * lda] = v;
        }
    }
}

cudaError_t symmetrize(double *A, int k, int64_t lda, cudaStream_t s)
{
    { count_launch(); symmetrize_kernel<<<256, 256, 0, s>>>(A, k, lda); }
    return cudaGetLastError();
}

__global__ void transpose_kernel(const double *A, double *B, int k)
{
    const int64_t total = (int64_t)k * k;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % k), j = (int)(e / k);
        B[j + (int64_t)i * k] = A[e];
    }
}

cudaError_t transpose_sq(const double *A, double *B, int k, cudaStream_t s)
{
    { count_launch(); transpose_kernel<<<256, 256, 0, s>>>(A, B, k); }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Vector steps of the Lanczos form of conjugate gradients (Algorithm 1)
// ---------------------------------------------------------------------------
// out[0] = x . y (one CTA of 1024 threads; n up to a few 10^5)
__global__ void __launch_bounds__(1024) dot1_kernel(int64_t n, const double *x, const double *y, double *out)
{
    __shared__ double red[32];
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s = fma(x[i], y[i], s);
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        double t = red[threadIdx.x];
        for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
        if (threadIdx.x == 0) out[0] = t;
    }
}

cudaError_t dot_dev(int64_t n, const double *x, const double *y, double *out, cudaStream_t s)
{
    count_launch();
    dot1_kernel<<<1, 1024, 0, s>>>(n, x, y, out);
    return cudaGetLastError();
}

// r = w - alpha[0] q - beta_prev qprev (qprev may be null)
__global__ void lanczos_resid_kernel(int64_t n, const double *w, const double *q, const double *qprev,
                                     const double *alpha, double beta_prev, double *r)
{
    const double a = *alpha;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        r[i] = w[i] - a * q[i] - (qprev ? beta_prev * qprev[i] : 0.0);
}

cudaError_t lanczos_resid(int64_t n, const double *w, const double *q, const double *qprev, const double *alpha,
                          double beta_prev, double *r, cudaStream_t s)
{
    count_launch();
    lanczos_resid_kernel<<<2 * num_sms(), 256, 0, s>>>(n, w, q, qprev, alpha, beta_prev, r);
    return cudaGetLastError();
}

// q = r / sqrt(rr[0])
__global__ void normalize_by_kernel(int64_t n, const double *r, const double *rr, double *q)
{
    const double inv = 1.0 / sqrt(*rr);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        q[i] = r[i] * inv;
}

cudaError_t normalize_by(int64_t n, const double *r, const double *rr, double *q, cudaStream_t s)
{
    count_launch();
    normalize_by_kernel<<<2 * num_sms(), 256, 0, s>>>(n, r, rr, q);
    return cudaGetLastError();
}

// T (m x m, column-major) = tridiag(beta[0..m-2], alpha[0..m-1], beta[0..m-2])
__global__ void tridiag_fill_kernel(int m, const double *alpha, const double *beta, double *T)
{
    const int64_t total = (int64_t)m * m;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % m), j = (int)(e / m);
        T[e] = (i == j) ? alpha[i] : ((i == j + 1 || j == i + 1) ? beta[i < j ? i : j] : 0.0);
    }
}

cudaError_t tridiag_fill(int m, const double *alpha, const double *beta, double *T, cudaStream_t s)
{
    count_launch();
    tridiag_fill_kernel<<<64, 256, 0, s>>>(m, alpha, beta, T);
    return cudaGetLastError();
}

// T (nb l x nb l, ld nb l) block tridiagonal from l x l blocks (column-major, ld l): diagonal
// block i = (M_i + M_i^T) / 2 with M_i at blocks + i l^2, block (i + 1, i) = W_i and block
// (i, i + 1) = W_i^T with W_i at blocks + (mcap + i) l^2
__global__ void block_tridiag_fill_kernel(int nb, int l, int mcap, const double *blocks, double *T)
{
    const int K = nb * l;
    const int64_t total = (int64_t)K * K;
    const int64_t ll = (int64_t)l * l;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(e % K), c = (int)(e / K);
        const int bi = r / l, bj = c / l, ri = r - bi * l, cj = c - bj * l;
        double v = 0.0;
        if (bi == bj) {
            const double *M = blocks + bi * ll;
            v = 0.5 * (M[ri + (int64_t)cj * l] + M[cj + (int64_t)ri * l]);
        } else if (bi == bj + 1) {
            v = blocks[(mcap + bj) * ll + ri + (int64_t)cj * l];
        } else if (bj == bi + 1) {
            v = blocks[(mcap + bi) * ll + cj + (int64_t)ri * l];
        }
        T[e] = v;
    }
}

cudaError_t block_tridiag_fill(int nb, int l, int mcap, const double *blocks, double *T, cudaStream_t s)
{
    if (nb < 1 || l < 1) return cudaSuccess;
    count_launch();
    block_tridiag_fill_kernel<<<128, 256, 0, s>>>(nb, l, mcap, blocks, T);
    return cudaGetLastError();
}

// c_i <- c_i / (1 + theta_i)
__global__ void div_one_plus_kernel(int m, double *c, const double *theta)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) c[i] /= 1.0 + theta[i];
}

cudaError_t div_one_plus(int m, double *c, const double *theta, cudaStream_t s)
{
    count_launch();
    div_one_plus_kernel<<<(m + 255) / 256, 256, 0, s>>>(m, c, theta);
    return cudaGetLastError();
}

__global__ void axpby_kernel(int64_t n, double a, const double *x, double b, double *y)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = a * x[i] + b * y[i];
}

cudaError_t axpby(int64_t n, double a, const double *x, double b, double *y, cudaStream_t s)
{
    int blocks = (int)((n + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) return cudaSuccess;
    { count_launch(); axpby_kernel<<<blocks, 256, 0, s>>>(n, a, x, b, y); }
    return cudaGetLastError();
}

// c_i <- -c_i / (1 + l_i) (LRA, smallest retained lambda > 1) or
// c_i <- c_i l_i / (1 + l_i) (LRU); mode written to mode_dev.
// Coefficients of the adaptive increment over the retained pairs: the leading m with
// lam_i >= rel_floor * lam_0 (all k when rel_floor < 0); mode_dev[0] = LRA (0) when the
// smallest retained eigenvalue is > 1, else LRU (1); mode_dev[1] = m.  Dropped pairs get
// coefficient 0 in either mode.
__global__ void increment_coef_kernel(const double *lam, int k, double *c, int *mode_dev, double rel_floor)
{
    __shared__ int m_s;
    if (threadIdx.x == 0) m_s = k;
    __syncthreads();
    if (rel_floor >= 0.0) {
        const double fl = rel_floor * lam[0];
        for (int i = threadIdx.x; i < k; i += blockDim.x)
            if (!(lam[i] >= fl)) atomicMin(&m_s, i);
    }
    __syncthreads();
    const int m = m_s > 0 ? m_s : 1;
    const int mode = (lam[m - 1] > 1.0) ? 0 : 1;
    for (int i = threadIdx.x; i < k; i += blockDim.x)
        c[i] = i >= m ? 0.0 : (mode == 0 ? -c[i] / (1.0 + lam[i]) : c[i] * lam[i] / (1.0 + lam[i]));
    if (threadIdx.x == 0) {
        mode_dev[0] = mode;
        mode_dev[1] = m;
    }
}

cudaError_t increment_coef(const double *lam, int k, double *c, int *mode_dev, double rel_floor, cudaStream_t s)
{
    { count_launch(); increment_coef_kernel<<<1, 1024, 0, s>>>(lam, k, c, mode_dev, rel_floor); }
    return cudaGetLastError();
}

__global__ void cov_coef_kernel(const double *lam, int m, double *coef, int *mode_dev)
{
    const int mode = (lam[m - 1] > 1.0) ? 0 : 1;
    for (int i = threadIdx.x; i < m; i += blockDim.x)
        coef[i] = mode == 0 ? 1.0 / (1.0 + lam[i]) : lam[i] / (1.0 + lam[i]);
    if (threadIdx.x == 0) mode_dev[0] = mode;
}

cudaError_t cov_coef(const double *lam, int m, double *coef, int *mode_dev, cudaStream_t s)
{
    { count_launch(); cov_coef_kernel<<<1, 1024, 0, s>>>(lam, m, coef, mode_dev); }
    return cudaGetLastError();
}

__global__ void check_finite_kernel(const double *x, int64_t n, int *flag)
{
    int bad = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (!isfinite(x[i])) bad = 1;
    if (bad) atomicOr(flag, 1);
}

__global__ void add_if_flag_kernel(const int *flag, int want, int64_t n, double a, const double *x, double *y)
{
    if (flag[0] != want) return;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] += a * x[i];
}

cudaError_t add_if_flag(const int *flag, int want, int64_t n, double a, const double *x, double *y, cudaStream_t s)
{
    int blocks = (int)((n + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) return cudaSuccess;
    { count_launch(); add_if_flag_kernel<<<blocks, 256, 0, s>>>(flag, want, n, a, x, y); }
    return cudaGetLastError();
}

__global__ void mul_kernel(int64_t n, const double *a, const double *b, double *out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = a[i] * b[i];
}

cudaError_t mul(int64_t n, const double *a, const double *b, double *out, cudaStream_t s)
{
    int blocks = (int)((n + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) return cudaSuccess;
    { count_launch(); mul_kernel<<<blocks, 256, 0, s>>>(n, a, b, out); }
    return cudaGetLastError();
}

// out[0] += 0.5 * sum x_i^2
__global__ void half_sq_kernel(int64_t n, const double *x, double *out)
{
    double part = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        part += x[i] * x[i];
    for (int off = 16; off > 0; off >>= 1) part += __shfl_down_sync(0xffffffffu, part, off);
    if ((threadIdx.x & 31) == 0 && part != 0.0) atomicAdd(out, 0.5 * part);
}

// out += 1/2 sum_o (d_o + r_o / rinv_o)^2 rinv_o: the observation term of the inner-loop
// quadratic cost (Eq. 3) from the innovation d and the tangent-linear residuals
// r = R^-1 H M L dv (rinv = 1 / sigma_o^2 > 0).
__global__ void obs_quad_kernel(int64_t p, const double *d, const double *r, const double *rinv, double *out)
{
    double part = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < p; i += (int64_t)gridDim.x * blockDim.x) {
        const double e = d[i] + (r ? r[i] / rinv[i] : 0.0);
        part += e * e * rinv[i];
    }
    for (int off = 16; off > 0; off >>= 1) part += __shfl_down_sync(0xffffffffu, part, off);
    if ((threadIdx.x & 31) == 0 && part != 0.0) atomicAdd(out, 0.5 * part);
}

// Column equilibration of a CholeskyQR pass: d_j = 1 / sqrt(G_jj) (1 for a
// zero column), G <- D G D on the lower triangle, Q <- Q D.  The scales are
// formed by their own kernel first: a block scaling its column must not race
// with another block still reading that column's diagonal entry.
__global__ void equil_scales_kernel(const double *G, int k, int64_t ldg, double *d)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= k) return;
    const double g = G[(int64_t)j * ldg + j];
    d[j] = g > 0.0 ? 1.0 / sqrt(g) : 1.0;
}

__global__ void equil_gram_kernel(double *G, int k, int64_t ldg, const double *d)
{
    const int col = blockIdx.x;
    if (col >= k) return;
    const double dc = d[col];
    for (int i = col + threadIdx.x; i < k; i += blockDim.x) G[(int64_t)col * ldg + i] *= d[i] * dc;
}

template <typename R>
__global__ void scale_cols_kernel(R *Q, int64_t n, int k, int64_t ldq, const double *d)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * k) return;
    const int64_t j = t / n, i = t - j * n;
    Q[j * ldq + i] = (R)((double)Q[j * ldq + i] * d[j]);
}

cudaError_t equilibrate(double *G, int k, int64_t ldg, void *Q, char tQ, int64_t n, int64_t ldq, double *d,
                        cudaStream_t s)
{
    if (k < 1) return cudaSuccess;
    count_launch();
    equil_scales_kernel<<<(k + 255) / 256, 256, 0, s>>>(G, k, ldg, d);
    count_launch();
    equil_gram_kernel<<<k, 256, 0, s>>>(G, k, ldg, d);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int64_t total = n * k;
    count_launch();
    if (tQ == 'd')
        scale_cols_kernel<double><<<(unsigned)((total + 255) / 256), 256, 0, s>>>((double *)Q, n, k, ldq, d);
    else
        scale_cols_kernel<float><<<(unsigned)((total + 255) / 256), 256, 0, s>>>((float *)Q, n, k, ldq, d);
    return cudaGetLastError();
}

__global__ void scale_to_f32_kernel(int64_t n, const double *in, double a, float *out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (float)(a * in[i]);
}

cudaError_t scale_to_f32(int64_t n, const double *in, double a, float *out, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    count_launch();
    scale_to_f32_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, in, a, out);
    return cudaGetLastError();
}

__global__ void scal_kernel(int64_t n, double a, double *x)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] *= a;
}

cudaError_t scal(int64_t n, double a, double *x, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    count_launch();
    scal_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, a, x);
    return cudaGetLastError();
}

// Y[j*ld + i] = a Y[j*ld + i] (+ W[j*ld + i]) for i < n, j < ncols (float or double)
template <typename R>
__global__ void scale_add_cols_kernel(int64_t n, int ncols, int64_t ld, R a, R *Y, const R *W)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * ncols) return;
    const int64_t j = t / n, i = t - j * n;
    const R v = a * Y[j * ld + i];
    Y[j * ld + i] = W ? v + W[j * ld + i] : v;
}

cudaError_t scale_add_cols(int64_t n, int ncols, int64_t ld, double a, void *Y, const void *W, int is_double,
                           cudaStream_t s)
{
    const int64_t total = n * ncols;
    if (total <= 0) return cudaSuccess;
    count_launch();
    const unsigned grid = (unsigned)((total + 255) / 256);
    if (is_double)
        scale_add_cols_kernel<double><<<grid, 256, 0, s>>>(n, ncols, ld, a, (double *)Y, (const double *)W);
    else
        scale_add_cols_kernel<float><<<grid, 256, 0, s>>>(n, ncols, ld, (float)a, (float *)Y, (const float *)W);
    return cudaGetLastError();
}

// T[j*ld + i] *= coef[i] for i < m, j < ncols (float or double block, FP64 coefficients)
template <typename R>
__global__ void scale_rows_kernel(int m, int ncols, int64_t ld, const double *__restrict__ coef, R *T)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)m * ncols) return;
    const int64_t j = t / m, i = t - j * m;
    T[j * ld + i] = (R)(coef[i] * (double)T[j * ld + i]);
}

cudaError_t scale_rows(int m, int ncols, int64_t ld, const double *coef, void *T, int is_double, cudaStream_t s)
{
    const int64_t total = (int64_t)m * ncols;
    if (total <= 0) return cudaSuccess;
    count_launch();
    const unsigned grid = (unsigned)((total + 255) / 256);
    if (is_double)
        scale_rows_kernel<double><<<grid, 256, 0, s>>>(m, ncols, ld, coef, (double *)T);
    else
        scale_rows_kernel<float><<<grid, 256, 0, s>>>(m, ncols, ld, coef, (float *)T);
    return cudaGetLastError();
}

// Y[j*ld + i] = a X[j*ld + i] + b Y[j*ld + i] for i < n, j < ncols (float or double)
template <typename R>
__global__ void axpby_cols_kernel(int64_t n, int ncols, int64_t ld, R a, const R *__restrict__ X, R b, R *Y)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * ncols) return;
    const int64_t j = t / n, i = t - j * n;
    Y[j * ld + i] = a * X[j * ld + i] + b * Y[j * ld + i];
}

cudaError_t axpby_cols(int64_t n, int ncols, int64_t ld, double a, const void *X, double b, void *Y, int is_double,
                       cudaStream_t s)
{
    const int64_t total = n * ncols;
    if (total <= 0) return cudaSuccess;
    count_launch();
    const unsigned grid = (unsigned)((total + 255) / 256);
    if (is_double)
        axpby_cols_kernel<double><<<grid, 256, 0, s>>>(n, ncols, ld, a, (const double *)X, b, (double *)Y);
    else
        axpby_cols_kernel<float><<<grid, 256, 0, s>>>(n, ncols, ld, (float)a, (const float *)X, (float)b, (float *)Y);
    return cudaGetLastError();
}

cudaError_t add_half_sq(int64_t n, const double *x, double *out, cudaStream_t s)
{
    int blocks = (int)((n + 255) / 256);
    if (blocks > 256) blocks = 256;
    if (blocks < 1) return cudaSuccess;
    { count_launch(); half_sq_kernel<<<blocks, 256, 0, s>>>(n, x, out); }
    return cudaGetLastError();
}

cudaError_t obs_quad_cost(int64_t p, const double *d, const double *r, const double *rinv, double *out, cudaStream_t s)
{
    int blocks = (int)((p + 255) / 256);
    if (blocks > 256) blocks = 256;
    if (blocks < 1) return cudaSuccess;
    { count_launch(); obs_quad_kernel<<<blocks, 256, 0, s>>>(p, d, r, rinv, out); }
    return cudaGetLastError();
}

// out[:, j] = in[:, perm[j]] for m columns of n doubles
__global__ void gather_cols_kernel(const double *in, int64_t ldi, const int *perm, int m, int64_t n, double *out,
                                   int64_t ldo)
{
    const int j = blockIdx.y;
    const double *src = in + (int64_t)perm[j] * ldi;
    double *dst = out + (int64_t)j * ldo;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[i];
}

cudaError_t gather_cols(const double *in, int64_t ldi, const int *perm, int m, int64_t n, double *out, int64_t ldo,
                        cudaStream_t s)
{
    if (m <= 0 || n <= 0) return cudaSuccess;
    int bx = (int)((n + 255) / 256);
    if (bx > 64) bx = 64;
    { count_launch(); gather_cols_kernel<<<dim3(bx, m), 256, 0, s>>>(in, ldi, perm, m, n, out, ldo); }
    return cudaGetLastError();
}

// Make the largest-magnitude entry of every column positive (first index on ties).
__global__ void fix_col_signs_kernel(double *U, int64_t n, int64_t ld)
{
    __shared__ double best_s[32];
    __shared__ int64_t bidx_s[32];
    double *u = U + (int64_t)blockIdx.x * ld;
    double best = -1.0;
    int64_t bidx = 0;
    for (int64_t r = threadIdx.x; r < n; r += blockDim.x) {
        const double v = fabs(u[r]);
        if (v > best) { best = v; bidx = r; }
    }
    for (int off = 16; off > 0; off >>= 1) {
        const double ob = __shfl_down_sync(0xffffffffu, best, off);
        const int64_t oi = __shfl_down_sync(0xffffffffu, bidx, off);
        if (ob > best || (ob == best && oi < bidx)) { best = ob; bidx = oi; }
    }
    if ((threadIdx.x & 31) == 0) { best_s[threadIdx.x >> 5] = best; bidx_s[threadIdx.x >> 5] = bidx; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x + 31) / 32; ++w)
            if (best_s[w] > best_s[0] || (best_s[w] == best_s[0] && bidx_s[w] < bidx_s[0])) {
                best_s[0] = best_s[w];
                bidx_s[0] = bidx_s[w];
            }
    }
    __syncthreads();
    if (u[bidx_s[0]] < 0.0)
        for (int64_t r = threadIdx.x; r < n; r += blockDim.x) u[r] = -u[r];
}

cudaError_t fix_col_signs(double *U, int64_t n, int k, int64_t ld, cudaStream_t s)
{
    if (k <= 0) return cudaSuccess;
    { count_launch(); fix_col_signs_kernel<<<k, 256, 0, s>>>(U, n, ld); }
    return cudaGetLastError();
}

cudaError_t check_finite(const double *x, int64_t n, int *flag, cudaStream_t s)
{
    int blocks = (int)((n + 255) / 256);
    if (blocks > 1024) blocks = 1024;
    if (blocks < 1) return cudaSuccess;
    { count_launch(); check_finite_kernel<<<blocks, 256, 0, s>>>(x, n, flag); }
    return cudaGetLastError();
}

}  // namespace riot
