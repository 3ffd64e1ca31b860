// FP32-accurate GEMM on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// C = alpha op(A) op(B) + beta C, column-major FP32 operands.  Each FP32
// value is split into three BF16 terms a = a1 + a2 + a3 (8 significant bits
// each, together the 24 of FP32), and the products a_i b_j with i + j <= 4
// (six tcgen05.mma per K step) are accumulated in FP32 in tensor memory: the
// result has FP32 accuracy at tensor-core speed.  This is how the sketch GEMMs
// of the randomized eigendecomposition (Q^T W, Q^T Y, U = Q Z) run in mixed
// precision.
//
// One CTA of 256 threads owns a 128 x 128 tile of C (its FP32 accumulator in
// 128 TMEM columns) and a slice of K (split-K over blockIdx.z, partial tiles
// reduced by a second kernel).  Per 64-wide K chunk the threads load the
// FP32 tiles (any transpose), split them and store the BF16 terms in shared
// memory in the canonical K-major core-matrix layout (8 rows x 16 bytes per
// core matrix, no swizzle), alternating between two stages; one thread issues
// the MMAs and commits them to the stage's mbarrier, which is waited on
// (bounded) before that stage is refilled.  The epilogue reads the
// accumulator with tcgen05.ld (each warp its 32 lanes, half the columns).
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace riot {

namespace {

constexpr int BM = 128, BN = 128, BK = 64;
constexpr int kThreads = 256;
constexpr int kSplits = 3;                         // BF16 terms per FP32 value
constexpr int kTileBytes = BM * BK * 2;            // one BF16 term of one operand tile (16 KB)
constexpr int kStageBytes = 2 * kSplits * kTileBytes;   // A and B terms of one K chunk (96 KB)
constexpr int kSmemBytes = 2 * kStageBytes + 1024;       // two stages

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: K-major, no swizzle.  LBO = byte distance
// between core matrices adjacent in K, SBO = between core matrices adjacent
// in M (or N); addresses and offsets in 16-byte units; bits 46-47 = 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor of kind::f16: D FP32, A and B BF16, both K-major, M x N.
__host__ __device__ constexpr uint32_t instr_desc(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Byte offset of element (r, k) of a 128 x 64 K-major tile in core-matrix
// layout: core (r / 8, k / 8) at ((k / 8) * 16 + r / 8) * 128, rows 16 bytes.
__device__ __forceinline__ uint32_t core_off(int r, int k)
{
    return (uint32_t)((((k >> 3) * 16 + (r >> 3)) << 7) + ((r & 7) << 4) + ((k & 7) << 1));
}

__device__ __forceinline__ void split3(float v, __nv_bfloat16 &a, __nv_bfloat16 &b, __nv_bfloat16 &c)
{
    a = __float2bfloat16(v);
    const float r1 = v - __bfloat162float(a);
    b = __float2bfloat16(r1);
    c = __float2bfloat16(r1 - __bfloat162float(b));
}

__device__ __forceinline__ void store_terms(const float (&v)[8], unsigned char *dst, uint32_t off)
{
    __align__(16) __nv_bfloat16 t[kSplits][8];
#pragma unroll
    for (int q = 0; q < 8; ++q) split3(v[q], t[0][q], t[1][q], t[2][q]);
#pragma unroll
    for (int s = 0; s < kSplits; ++s)
        *reinterpret_cast<uint4 *>(dst + s * kTileBytes + off) = *reinterpret_cast<const uint4 *>(t[s]);
}

// Load a 128 x 64 tile of X (element (r, k) at X[k + r ld] when k_contig, else
// X[r + k ld]), rows r0.., k0.., zero outside rows x kvalid, split into three
// BF16 terms stored at dst + s * kTileBytes.  Each thread handles runs of 8 k
// of one row (one core-matrix row); the eight threads that store neighbouring
// 16-byte rows of a core matrix are consecutive, so the stores do not conflict.
__device__ __forceinline__ void load_tile(const float *X, long long ld, bool k_contig, int r0, int rows, int k0,
                                          int kvalid, unsigned char *dst)
{
    const int tid = threadIdx.x;
    if (k_contig) {
        // tid = (kq8, rg, rr): rr = row within 8, kq8 = 8-wide k run, 4 row groups per pass
        const int rr = tid & 7, kq = ((tid >> 3) & 7) * 8, rg = tid >> 6;
        for (int p = 0; p < BM / 32; ++p) {
            const int r = p * 32 + rg * 8 + rr;
            const int gr = r0 + r;
            float v[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int gk = k0 + kq + q;
                v[q] = (gr < rows && gk < kvalid) ? X[(long long)gk + (long long)gr * ld] : 0.f;
            }
            store_terms(v, dst, core_off(r, kq));
        }
    } else {
        // one row per thread, rows contiguous in memory across the warp; two halves of k
        const int r = tid & (BM - 1), kh = (tid >> 7) * (BK / 2);
        const int gr = r0 + r;
        for (int kq = kh; kq < kh + BK / 2; kq += 8) {
            float v[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int gk = k0 + kq + q;
                v[q] = (gr < rows && gk < kvalid) ? X[(long long)gr + (long long)gk * ld] : 0.f;
            }
            store_terms(v, dst, core_off(r, kq));
        }
    }
}

__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity)
{
    for (int i = 0; i < (1 << 22); ++i) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
        if (i > 64) __nanosleep(32);
    }
    return false;
}

struct TcArgs {
    const float *A, *B;
    float *C;          // output (the workspace when split: slice z at C + z * cslice)
    long long lda, ldb, ldc, cslice;
    int M, N, K, kchunk;
    int a_kcontig, b_kcontig;
    float alpha, beta;  // applied here only when not split
    int *err;
};

// Two shared-memory stages: while the tensor cores multiply chunk c, the
// threads load and split chunk c + 1 into the other stage; a stage is
// refilled only after the mbarrier committed with its MMAs has completed.
__global__ void __launch_bounds__(kThreads, 1) tc_gemm_kernel(TcArgs g)
{
    extern __shared__ __align__(1024) unsigned char smem_dyn[];
    unsigned char *base = reinterpret_cast<unsigned char *>(((uintptr_t)smem_dyn + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ uint32_t tmem_holder;
    __shared__ int abort_s;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
    const int kbeg = blockIdx.z * g.kchunk;
    const int kend = min(g.K, kbeg + g.kchunk);
    const int nchunks = kend > kbeg ? (kend - kbeg + BK - 1) / BK : 0;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_holder)),
                     "r"(BN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        abort_s = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bars[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bars[1])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_holder;
    constexpr uint32_t idesc = instr_desc(BM, BN);
    float *C = g.C + (long long)blockIdx.z * g.cslice;
    uint32_t ph[2] = {0u, 0u};   // parity of the next completion of each stage's barrier (thread 0)
    for (int c = 0; c < nchunks; ++c) {
        const int st = c & 1;
        unsigned char *sA = base + st * kStageBytes;
        unsigned char *sB = sA + kSplits * kTileBytes;
        if (c >= 2) {
            // this stage still feeds the MMAs of chunk c - 2
            if (tid == 0 && !abort_s) {
                if (!mbar_wait_bounded(smem_u32(&bars[st]), ph[st])) {
                    abort_s = 1;
                    atomicExch(g.err, 1);
                }
                ph[st] ^= 1u;
            }
            __syncthreads();
        }
        const int k0 = kbeg + c * BK;
        load_tile(g.A, g.lda, g.a_kcontig, m0, g.M, k0, kend, sA);
        load_tile(g.B, g.ldb, g.b_kcontig, n0, g.N, k0, kend, sB);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0 && !abort_s) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            // products a_i b_j with i + j <= 4 (terms counted from 1)
            const int pa[6] = {0, 0, 1, 0, 1, 2};
            const int pb[6] = {0, 1, 0, 2, 1, 0};
#pragma unroll
            for (int ks = 0; ks < BK / 16; ++ks) {
#pragma unroll
                for (int p = 0; p < 6; ++p) {
                    const uint32_t a_addr = smem_u32(sA + pa[p] * kTileBytes) + ks * 4096;
                    const uint32_t b_addr = smem_u32(sB + pb[p] * kTileBytes) + ks * 4096;
                    const uint64_t ad = smem_desc(a_addr, 2048, 128);
                    const uint64_t bd = smem_desc(b_addr, 2048, 128);
                    const uint32_t acc = (c > 0 || ks > 0 || p > 0) ? 1u : 0u;
                    asm volatile(
                        "{\n\t.reg .pred p;\n\t"
                        "setp.ne.b32 p, %4, 0;\n\t"
                        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                        "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                        : "memory");
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&bars[st]))
                         : "memory");
        }
    }
    // wait for the MMAs still in flight (the last two chunks)
    if (tid == 0 && !abort_s) {
        for (int c = (nchunks >= 2 ? nchunks - 2 : 0); c < nchunks; ++c) {
            const int st = c & 1;
            if (!mbar_wait_bounded(smem_u32(&bars[st]), ph[st])) {
                abort_s = 1;
                atomicExch(g.err, 1);
                break;
            }
            ph[st] ^= 1u;
        }
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // epilogue: warp w reads lanes 32 (w % 4) .. + 31 (rows); warps 0-3 columns 0-63, 4-7 columns 64-127
    const int row = m0 + (warp & 3) * 32 + (tid & 31);
    const int cbeg = (warp >> 2) * (BN / 2);
    for (int c0 = cbeg; c0 < cbeg + BN / 2; c0 += 32) {
        uint32_t r[32];
        const uint32_t taddr = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)c0;
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
            "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
              "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
              "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (row < g.M) {
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const int col = n0 + c0 + j;
                if (col < g.N) {
                    float *p = C + row + (long long)col * g.ldc;
                    const float v = nchunks > 0 ? __uint_as_float(r[j]) : 0.f;
                    *p = g.alpha * v + (g.beta != 0.f ? g.beta * *p : 0.f);
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN) : "memory");
}

__global__ void sum_splits_kernel(const float *ws, int S, int M, int N, float alpha, float beta, float *C, long long ldc)
{
    const long long total = (long long)M * N;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e % M), j = (int)(e / M);
        float s = 0.f;
        for (int z = 0; z < S; ++z) s += ws[(long long)z * total + e];
        float *p = C + i + (long long)j * ldc;
        *p = alpha * s + (beta != 0.f ? beta * *p : 0.f);
    }
}


// ---------------------------------------------------------------------------
// G = Y^T Y of an FP32 block Y (n x k) to FP64-level accuracy on the tensor
// cores, by error-free splitting (Ozaki, Ogita, Oishi and Rump 2012):
// column j is scaled by 2^-e_j (|y| < 2^e_j) and split into five integer
// slices of 8, 7, 7, 7 and 7 bits,
//     y = 2^e_j (s1 2^-7 + s2 2^-14 + s3 2^-21 + s4 2^-28 + s5 2^-35) + r,
//     |r| <= 2^(e_j - 36),
// |s1| <= 128, |s2..5| <= 64, each exact in BF16.  A product of two slices is
// an integer below 2^14 in magnitude; slice pairs (a, b) of equal weight
// 2^-7(a+b) share one FP32 accumulator in tensor memory (w = a + b = 2..6:
// 1 to 5 pairs, five accumulators of 64 columns for a 128 x 64 tile of G), and
// a K range of at most kGramMaxKR rows keeps every partial sum of every
// accumulator below 2^23, so the tensor-core accumulation is exact.  The
// epilogue combines the five integers in 64-bit arithmetic and adds its K
// range's part atomically into an int64 Gram; a last kernel scales that by
// 2^(e_i + e_j - 42) into FP64.  What is dropped (pairs with w >= 7, the
// residuals r) is below about 2^-35 of max|y_i| max|y_j| per row of Y and of
// random sign off the diagonal; on the diagonal the dropped s4^2 terms all
// have the same sign, so the diagonal is summed in FP64 on the CUDA cores
// instead (n k FMAs, next to the column maxima).
// ---------------------------------------------------------------------------
constexpr int kGramBK = 32;                            // K rows per chunk
constexpr int kGramBN = 64;                            // columns of a Gram tile
constexpr int kGramSlices = 5;
constexpr int kGramPairs = kGramSlices * (kGramSlices + 1) / 2;     // pairs with a + b <= 6 (1-based)
constexpr int kGramTileBytes = BM * kGramBK * 2;       // one slice of one operand, 128-row layout (8 KB)
constexpr int kGramStageBytes = 2 * kGramSlices * kGramTileBytes;   // 80 KB
constexpr int kGramSmemBytes = 2 * kGramStageBytes + 1024;
constexpr int kGramMaxKR = 288;                        // 288 * 7 * 2^12 < 2^23
constexpr int kGramAccCols = 512;                      // five accumulators of 64 columns (allocation: a power of 2)
constexpr int kGramNonFinite = -100000;                // exponent of a column with Inf or NaN

// Exponent e (max |y| < 2^e), the two power-of-two factors f1 f2 = 2^(7 - e)
// (two so that both stay normal FP32 numbers) and the FP64 sum of squares of
// each column.
__global__ void gram_colscale_kernel(const float *Y, int n, int k, long long ldy, int *colexp, float2 *colscale,
                                     double *coldiag)
{
    const int j = blockIdx.x;
    if (j >= k) return;
    const float *y = Y + (long long)j * ldy;
    float m = 0.f;
    double ss = 0.0;
    int bad = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const float v = y[i];
        bad |= !isfinite(v);
        m = fmaxf(m, fabsf(v));
        ss = fma((double)v, (double)v, ss);
    }
    __shared__ float red[32];
    __shared__ double reds[32];
    for (int off = 16; off > 0; off >>= 1) {
        m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
        ss += __shfl_xor_sync(0xffffffffu, ss, off);
    }
    if ((threadIdx.x & 31) == 0) {
        red[threadIdx.x >> 5] = m;
        reds[threadIdx.x >> 5] = ss;
    }
    bad = __syncthreads_or(bad);
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
            m = fmaxf(m, red[w]);
            ss += reds[w];
        }
        coldiag[j] = bad ? __longlong_as_double(0x7ff8000000000000LL) : ss;
        int e = 0;
        if (m > 0.f) frexpf(m, &e);   // m = f 2^e, f in [0.5, 1)
        const int se = 7 - e, x1 = se < 127 ? se : 127, x2 = se - x1;
        colexp[j] = bad ? kGramNonFinite : e;
        colscale[j] = bad ? make_float2(0.f, 0.f)
                          : make_float2(__int_as_float((127 + x1) << 23), __int_as_float((127 + x2) << 23));
    }
}

__device__ __forceinline__ void slice5(float y, float2 f, float (&s)[kGramSlices])
{
    float t = (y * f.x) * f.y;   // |t| < 128, exact
#pragma unroll
    for (int q = 0; q < kGramSlices; ++q) {
        s[q] = rintf(t);
        t = (t - s[q]) * 128.f;  // exact: t - s is the fraction left over
    }
}

// Rows r0 .. r0 + ROWS - 1 of the Gram (columns of Y), K rows k0 .. k0 + 31,
// in the 128-row core-matrix layout: element (r, l) is Y[l + r ldy]; each
// thread handles runs of 8 l of one row.
template <int ROWS>
__device__ __forceinline__ void gram_load_tile(const float *Y, long long ldy, int r0, int k, int k0, int kend,
                                               const float2 *colscale, unsigned char *dst)
{
    const int tid = threadIdx.x;
    const int rr = tid & 7, kq = ((tid >> 3) & 3) * 8, rg = tid >> 5;
#pragma unroll
    for (int p = 0; p < ROWS / 64; ++p) {
        const int r = p * 64 + rg * 8 + rr;
        const int gr = r0 + r;
        const float2 f = (gr < k) ? colscale[gr] : make_float2(0.f, 0.f);
        __align__(16) __nv_bfloat16 t[kGramSlices][8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int gl = k0 + kq + q;
            const float v = (gr < k && gl < kend) ? Y[(long long)gl + (long long)gr * ldy] : 0.f;
            float s[kGramSlices];
            slice5(v, f, s);
#pragma unroll
            for (int z = 0; z < kGramSlices; ++z) t[z][q] = __float2bfloat16_rn(s[z]);
        }
        const uint32_t off = core_off(r, kq);
#pragma unroll
        for (int z = 0; z < kGramSlices; ++z)
            *reinterpret_cast<uint4 *>(dst + z * kGramTileBytes + off) = *reinterpret_cast<const uint4 *>(t[z]);
    }
}

struct GramArgs {
    const float *Y;
    long long ldy;
    int n, k, kr;               // rows of Y, columns of Y, K rows per split
    const float2 *colscale;
    unsigned long long *acc;    // k x k int64 Gram (two's complement), column-major
    int *err;
};

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}

// blockIdx.x = tile (ti, tj) of 128 rows x 64 columns reaching the lower triangle
// (tj <= 2 ti + 1), row by row; blockIdx.y = K split.
__global__ void __launch_bounds__(kThreads, 1) tc_gram_kernel(GramArgs g)
{
    extern __shared__ __align__(1024) unsigned char smem_dyn[];
    unsigned char *base = reinterpret_cast<unsigned char *>(((uintptr_t)smem_dyn + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ uint32_t tmem_holder;
    __shared__ int abort_s;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int tk2 = (g.k + kGramBN - 1) / kGramBN;
    int ti = 0, rem = blockIdx.x;
    while (rem >= min(2 * ti + 2, tk2)) { rem -= min(2 * ti + 2, tk2); ++ti; }
    const int tj = rem;
    const bool diag = (tj >= 2 * ti);     // the tile's columns are rows of its own A tile
    const int m0 = ti * BM, n0 = tj * kGramBN;
    const int kbeg = blockIdx.y * g.kr;
    const int kend = min(g.n, kbeg + g.kr);
    const int nchunks = kend > kbeg ? (kend - kbeg + kGramBK - 1) / kGramBK : 0;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_holder)),
                     "r"(kGramAccCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        abort_s = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bars[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bars[1])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_holder;
    constexpr uint32_t idesc = instr_desc(BM, kGramBN);
    uint32_t ph[2] = {0u, 0u};
    for (int c = 0; c < nchunks; ++c) {
        const int st = c & 1;
        unsigned char *sA = base + st * kGramStageBytes;
        unsigned char *sB = diag ? sA + (tj - 2 * ti) * 1024 : sA + kGramSlices * kGramTileBytes;
        if (c >= 2) {
            if (tid == 0 && !abort_s) {
                if (!mbar_wait_bounded(smem_u32(&bars[st]), ph[st])) {
                    abort_s = 1;
                    atomicExch(g.err, 1);
                }
                ph[st] ^= 1u;
            }
            __syncthreads();
        }
        const int k0 = kbeg + c * kGramBK;
        gram_load_tile<BM>(g.Y, g.ldy, m0, g.k, k0, kend, g.colscale, sA);
        if (!diag) gram_load_tile<kGramBN>(g.Y, g.ldy, n0, g.k, k0, kend, g.colscale, sB);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0 && !abort_s) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            // slice pairs (a, b), 0-based, grouped by weight a + b = 0 .. 4 (accumulator a + b)
            const int pa[kGramPairs] = {0, 0, 1, 0, 1, 2, 0, 1, 2, 3, 0, 1, 2, 3, 4};
            const int pb[kGramPairs] = {0, 1, 0, 2, 1, 0, 3, 2, 1, 0, 4, 3, 2, 1, 0};
#pragma unroll
            for (int ks = 0; ks < kGramBK / 16; ++ks) {
#pragma unroll
                for (int p = 0; p < kGramPairs; ++p) {
                    const int w = pa[p] + pb[p];
                    const bool first_of_group = (pa[p] == 0);
                    const uint32_t a_addr = smem_u32(sA + pa[p] * kGramTileBytes) + ks * 4096;
                    const uint32_t b_addr = smem_u32(sB + pb[p] * kGramTileBytes) + ks * 4096;
                    const uint64_t ad = smem_desc(a_addr, 2048, 128);
                    const uint64_t bd = smem_desc(b_addr, 2048, 128);
                    const uint32_t acc = (c > 0 || ks > 0 || !first_of_group) ? 1u : 0u;
                    asm volatile(
                        "{\n\t.reg .pred p;\n\t"
                        "setp.ne.b32 p, %4, 0;\n\t"
                        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem + (uint32_t)(w * kGramBN)),
                        "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                        : "memory");
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&bars[st]))
                         : "memory");
        }
    }
    if (tid == 0 && !abort_s) {
        for (int c = (nchunks >= 2 ? nchunks - 2 : 0); c < nchunks; ++c) {
            const int st = c & 1;
            if (!mbar_wait_bounded(smem_u32(&bars[st]), ph[st])) {
                abort_s = 1;
                atomicExch(g.err, 1);
                break;
            }
            ph[st] ^= 1u;
        }
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // epilogue: warp w reads TMEM lanes 32 (w % 4) ..; warps 0-3 columns 0-31, warps 4-7 columns 32-63
    const int row = m0 + (warp & 3) * 32 + (tid & 31);
    const int cbeg = (warp >> 2) * (kGramBN / 2);
    if (nchunks > 0 && !abort_s) {
        for (int c0 = cbeg; c0 < cbeg + kGramBN / 2; c0 += 16) {
            uint32_t r[kGramSlices][16];
            const uint32_t taddr = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)c0;
#pragma unroll
            for (int w = 0; w < kGramSlices; ++w) tmem_ld16(taddr + (uint32_t)(w * kGramBN), r[w]);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (row < g.k) {
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const int col = n0 + c0 + q;
                    if (col < g.k && col < row) {
                        long long t = 0;
#pragma unroll
                        for (int w = 0; w < kGramSlices; ++w)
                            t += (long long)__float2int_rn(__uint_as_float(r[w][q])) << (7 * (kGramSlices - 1 - w));
                        atomicAdd(g.acc + row + (long long)col * g.k, (unsigned long long)t);
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kGramAccCols) : "memory");
}

// G (strict lower triangle) = int64 Gram * 2^(e_i + e_j - 42), the diagonal from the FP64
// column sums; NaN where a column held Inf or NaN.
__global__ void gram_finish_kernel(const unsigned long long *acc, const int *colexp, const double *coldiag, int k,
                                   double *G, long long ldg)
{
    const long long total = (long long)k * k;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e % k), j = (int)(e / k);
        if (i < j) continue;
        const int ei = colexp[i], ej = colexp[j];
        double v;
        if (ei == kGramNonFinite || ej == kGramNonFinite) v = __longlong_as_double(0x7ff8000000000000LL);
        else if (i == j) v = coldiag[i];
        else v = ldexp((double)(long long)acc[e], ei + ej - 42);
        G[i + (long long)j * ldg] = v;
    }
}

}  // namespace

size_t tc_sgemm_ws_floats(int m, int n, int k)
{
    const int tiles = ((m + BM - 1) / BM) * ((n + BN - 1) / BN);
    int S = (num_sms() + tiles - 1) / tiles;
    const int kchunks = (k + BK - 1) / BK;
    if (S > kchunks) S = kchunks;
    if (S > 16) S = 16;
    return S > 1 ? (size_t)S * m * n : 0;
}

cudaError_t tc_sgemm(char ta, char tb, int m, int n, int k, float alpha, const float *A, int64_t lda, const float *B,
                     int64_t ldb, float beta, float *C, int64_t ldc, float *ws, size_t ws_floats, int *err,
                     cudaStream_t s)
{
    if (m <= 0 || n <= 0) return cudaSuccess;
    static bool attr_done = false;
    if (!attr_done) {
        cudaError_t e = cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
        if (e != cudaSuccess) return e;
        attr_done = true;
    }
    const int tiles_m = (m + BM - 1) / BM, tiles_n = (n + BN - 1) / BN;
    int S = (num_sms() + tiles_m * tiles_n - 1) / (tiles_m * tiles_n);
    const int kchunks = (k + BK - 1) / BK;
    if (S > kchunks) S = kchunks;
    if (S > 16) S = 16;
    if (S < 1) S = 1;
    while (S > 1 && (!ws || (size_t)S * m * n > ws_floats)) --S;
    const int kc = ((kchunks + S - 1) / S) * BK;
    S = (k + kc - 1) / kc;
    if (S < 1) S = 1;
    TcArgs g;
    g.A = A;
    g.B = B;
    g.lda = lda;
    g.ldb = ldb;
    g.M = m;
    g.N = n;
    g.K = k;
    g.kchunk = kc > 0 ? kc : BK;
    g.a_kcontig = (ta == 'T');
    g.b_kcontig = (tb != 'T');
    g.err = err;
    if (S == 1) {
        g.C = C;
        g.ldc = ldc;
        g.cslice = 0;
        g.alpha = alpha;
        g.beta = beta;
    } else {
        g.C = ws;
        g.ldc = m;
        g.cslice = (long long)m * n;
        g.alpha = 1.f;
        g.beta = 0.f;
    }
    dim3 grid(tiles_m, tiles_n, S);
    count_launch();
    tc_gemm_kernel<<<grid, kThreads, kSmemBytes, s>>>(g);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || S == 1) return e;
    count_launch();
    sum_splits_kernel<<<256, 256, 0, s>>>(ws, S, m, n, alpha, beta, C, ldc);
    return cudaGetLastError();
}

size_t tc_gram_ws_bytes(int k)
{
    return (size_t)k * k * sizeof(unsigned long long) + (size_t)k * (sizeof(int) + sizeof(float2) + sizeof(double)) +
           64;
}

cudaError_t tc_gram_f32(int n, int k, const float *Y, int64_t ldy, double *G, int64_t ldg, void *ws, int *err,
                        cudaStream_t s)
{
    if (k <= 0) return cudaSuccess;
    static bool attr_done = false;
    if (!attr_done) {
        cudaError_t e = cudaFuncSetAttribute(tc_gram_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             kGramSmemBytes);
        if (e != cudaSuccess) return e;
        attr_done = true;
    }
    unsigned long long *acc = (unsigned long long *)ws;
    int *colexp = (int *)(acc + (size_t)k * k);
    float2 *colscale = (float2 *)(((uintptr_t)(colexp + k) + 15) & ~(uintptr_t)15);
    double *coldiag = (double *)(colscale + k);
    cudaError_t e = cudaMemsetAsync(acc, 0, (size_t)k * k * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    count_launch();
    gram_colscale_kernel<<<k, 256, 0, s>>>(Y, n, k, ldy, colexp, colscale, coldiag);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int tk = (k + BM - 1) / BM, tk2 = (k + kGramBN - 1) / kGramBN;
    int tiles = 0;
    for (int ti = 0; ti < tk; ++ti) tiles += (2 * ti + 2 < tk2) ? 2 * ti + 2 : tk2;
    // K splits: as many as fill the GPU once, each at most kGramMaxKR rows (exactness bound)
    int S = num_sms() / tiles;
    if (S < 1) S = 1;
    int kr = ((n + S - 1) / S + kGramBK - 1) / kGramBK * kGramBK;
    if (kr > kGramMaxKR) kr = kGramMaxKR;
    if (kr < kGramBK) kr = kGramBK;
    S = n > 0 ? (n + kr - 1) / kr : 1;
    GramArgs g;
    g.Y = Y;
    g.ldy = ldy;
    g.n = n;
    g.k = k;
    g.kr = kr;
    g.colscale = colscale;
    g.acc = acc;
    g.err = err;
    count_launch();
    tc_gram_kernel<<<dim3(tiles, S), kThreads, kGramSmemBytes, s>>>(g);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    count_launch();
    gram_finish_kernel<<<2 * num_sms(), 256, 0, s>>>(acc, colexp, coldiag, k, G, ldg);
    return cudaGetLastError();
}

}  // namespace riot
