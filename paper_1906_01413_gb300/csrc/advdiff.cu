// Tracer transport of the surface-emission inversion (the setting of the
// paper's black-carbon experiments, Section 3.2, on a synthetic box model):
// batched RK4 tangent-linear and adjoint steppers, trilinear observation
// gather / scatter, and the separable exponential prior square root.
//
// Stepper design.  One launch advances a batch of sketch columns ("probes")
// by one RK4 step.  A CTA owns a TX x TY tile of columns (x, y) of one probe,
// every level, plus a halo of 4 columns on each side: the four RK4 stages are
// computed on chip, each on a region one column narrower than the last
// (stage s is valid on the tile grown by 4 - s), so the state is read once
// and written once per step.  A thread owns one column of the region and
// keeps its levels in registers (step input, stage input, RK4 accumulator);
// the horizontal neighbours of a stage input come from one shared-memory
// plane per level, the vertical ones from the thread's own registers.  The
// upwind advection of a column reduces to five coefficients (self and the
// four neighbours) computed once from the face winds and scaled per level;
// the adjoint uses the transposed coefficients, so the same kernel steps
// both directions.  For a linear autonomous system the RK4 step is
// c+ = P(hA) c + h Q(hA) s, and its adjoint gives the source adjoint
// h Q(hA^T) lam = h/6 (lam + 2 u1 + 2 u2 + u3) from the adjoint stage inputs
// u1..u3, accumulated at level 0 for the emission blocks.
#include <cuda_runtime.h>
#include <math.h>

#include "internal.h"

namespace riot {

namespace {

constexpr int kHalo = 4;

constexpr int kMaxNZ = 32;

template <typename R>
struct StepArgs {
    R amp[kMaxNZ];        // level scaling of the winds (0 beyond nz)
    R kzs[kMaxNZ + 1];    // Kz / dz^2 on face l-1/2 (0 on the bottom, the top and beyond)
    const R *cin;
    R *cout;
    long long pstride;    // cells per probe
    const R *src;         // surface source of this step's block (TL), per probe at sstride
    long long sstride;
    R *ebar;              // source adjoint of this step's block (AD), per probe at estride
    long long estride;
    const R *u, *v;
    int nx, ny, nz;
    R h, rdx, rdy;
};

template <typename R, int NZ, int TX, int TY, bool ADJ>
__global__ void __launch_bounds__((TX + 2 * kHalo) * (TY + 2 * kHalo), 1) adv_step_kernel(StepArgs<R> a)
{
    constexpr int RX = TX + 2 * kHalo, RY = TY + 2 * kHalo, PL = RX * RY;
    extern __shared__ __align__(16) unsigned char adv_smem[];
    // two [NZ][RY][RX] planes of stage inputs, used alternately: one barrier per stage
    R *S0 = reinterpret_cast<R *>(adv_smem);
    const int tid = threadIdx.x;
    const int rx = tid % RX, ry = tid / RX;
    const int nx = a.nx, ny = a.ny;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    int gx = (x0 - kHalo + rx) % nx;
    if (gx < 0) gx += nx;
    const int gy = y0 - kHalo + ry;
    const bool valid = gy >= 0 && gy < ny;
    const size_t plane = (size_t)nx * ny;
    const size_t col = valid ? (size_t)gy * nx + gx : 0;
    // advection coefficients of this column at amplitude 1 (1/s)
    R c0 = 0, cE = 0, cW = 0, cN = 0, cS = 0;
    if (valid) {
        const R uL = a.u[col], uR = a.u[(size_t)gy * nx + (gx + 1 == nx ? 0 : gx + 1)];
        const R vS = a.v[col], vN = a.v[col + nx];
        const R z0 = R(0);
        const R uLp = uL > z0 ? uL : z0, uLm = uL < z0 ? uL : z0;
        const R uRp = uR > z0 ? uR : z0, uRm = uR < z0 ? uR : z0;
        const R vSp = vS > z0 ? vS : z0, vSm = vS < z0 ? vS : z0;
        const R vNp = vN > z0 ? vN : z0, vNm = vN < z0 ? vN : z0;
        c0 = (uLm - uRp) * a.rdx + (vSm - vNp) * a.rdy;
        if (!ADJ) {
            cE = -uRm * a.rdx;
            cW = uLp * a.rdx;
            cN = -vNm * a.rdy;
            cS = vSp * a.rdy;
        } else {
            cE = uRp * a.rdx;
            cW = -uLm * a.rdx;
            cN = vNp * a.rdy;
            cS = -vSm * a.rdy;
        }
    }
    const size_t pb = (size_t)blockIdx.z * a.pstride;
    R c[NZ], w[NZ], acc[NZ];
#pragma unroll
    for (int z = 0; z < NZ; ++z) {
        c[z] = (valid && z < a.nz) ? a.cin[pb + z * plane + col] : R(0);
        w[z] = c[z];
        acc[z] = R(0);
    }
    R s0 = R(0);
    if (!ADJ && valid && a.src) s0 = a.src[(size_t)blockIdx.z * a.sstride + col];
    const R h = a.h, h2 = R(0.5) * a.h, h3 = a.h / R(3), h6 = a.h / R(6);
    R e0 = R(0);
#pragma unroll
    for (int st = 1; st <= 4; ++st) {
        R *S = S0 + (st & 1) * NZ * PL;
        // the stage input is read on the region of this stage grown by one column;
        // rows beyond the walls publish their zeros (their coefficients are 0, but
        // a stale value times 0 would not be)
        const bool pub = rx >= st - 1 && rx < RX - st + 1 && ry >= st - 1 && ry < RY - st + 1;
        if (pub) {
#pragma unroll
            for (int z = 0; z < NZ; ++z) S[z * PL + ry * RX + rx] = w[z];
        }
        if (ADJ) e0 += (st == 1 || st == 4) ? w[0] : R(2) * w[0];
        __syncthreads();
        const bool act = valid && rx >= st && rx < RX - st && ry >= st && ry < RY - st;
        if (act) {
            R wm = R(0);
#pragma unroll
            for (int z = 0; z < NZ; ++z) {
                const R wz = w[z];
                const R wp = (z + 1 < NZ) ? w[z + 1] : R(0);
                const R *Sz = S + z * PL + ry * RX + rx;
                const R hor = c0 * wz + cE * Sz[1] + cW * Sz[-1] + cN * Sz[RX] + cS * Sz[-RX];
                R k = a.amp[z] * hor + a.kzs[z + 1] * (wp - wz) - a.kzs[z] * (wz - wm);
                if (!ADJ && z == 0) k += s0;
                if (st == 1) {
                    acc[z] = c[z] + h6 * k;
                    w[z] = c[z] + h2 * k;
                } else if (st == 2) {
                    acc[z] += h3 * k;
                    w[z] = c[z] + h2 * k;
                } else if (st == 3) {
                    acc[z] += h3 * k;
                    w[z] = c[z] + h * k;
                } else {
                    acc[z] += h6 * k;
                }
                wm = wz;
            }
        }
    }
    const int ix = rx - kHalo, iy = ry - kHalo;
    if (valid && ix >= 0 && ix < TX && iy >= 0 && iy < TY && x0 + ix < nx) {
#pragma unroll
        for (int z = 0; z < NZ; ++z)
            if (z < a.nz) a.cout[pb + z * plane + col] = acc[z];
        if (ADJ && a.ebar) a.ebar[(size_t)blockIdx.z * a.estride + col] += h6 * e0;
    }
}

// FP32 stepper: nested RK4 on pairs of levels with packed FP32x2 arithmetic.  For the
// linear autonomous tendency f(w) = A w + s of one step, RK4 gives c+ = P(hA) c + h Q(hA) s,
// P and Q the Taylor polynomials of degree 4 and 3 of exp(z) and (exp(z) - 1) / z.  Nested
// (Horner), that is w <- c + a (A w + s) for a = h/4, h/3, h/2, h from w = c, the last w being
// c+: the same four applications of A as the classical stages, with one state array besides
// c instead of two.  The adjoint P(hA^T) lam is the same recursion with A^T and no source;
// the input of its last stage is Q(hA^T) lam, so the source adjoint is h times its level 0.
// Levels are held in pairs (2p, 2p + 1) (padded with zero coefficients beyond nz) and
// combined by packed FP32x2 instructions, one instruction for two levels; the shared planes
// hold the pairs, so a horizontal neighbour fetch is one 64-bit load for two levels.  (Pairs
// (p, p + NZP), whose vertical neighbours are whole pairs, measured slower: the renamed
// stage inputs cost registers.)  Tiles and halo as in adv_step_kernel.
struct StepArgsF2 {
    float2 amp2[16];   // (amp of level 2p, of level 2p + 1); 0 beyond nz
    float2 ku2[16];    // Kz / dz^2 on the face above each level of the pair
    float2 kl2[16];    // on the face below
    float2 nkd2[16];   // -(ku + kl)
    const float *cin;
    float *cout;
    long long pstride;
    const float *src;
    long long sstride;
    float *ebar;
    long long estride;
    const float *u, *v;
    int nx, ny, nz;
    float h, rdx, rdy;
};

// registers per thread that still fit one CTA of `threads` on an SM (registers go to warps in
// groups of four, in steps of 8 per thread)
constexpr int regs_for(int threads)
{
    return ((65536 / ((threads + 127) / 128 * 128)) / 8 * 8) > 255 ? 255 : (65536 / ((threads + 127) / 128 * 128)) / 8 * 8;
}

template <int NZP, int TX, int TY, bool ADJ>
__global__ void __maxnreg__(regs_for((TX + 2 * kHalo) * (TY + 2 * kHalo))) adv_step_f2_kernel(StepArgsF2 a)
{
    constexpr int RX = TX + 2 * kHalo, RY = TY + 2 * kHalo, PL = RX * RY;
    extern __shared__ __align__(16) unsigned char adv2_smem[];
    float2 *S0 = reinterpret_cast<float2 *>(adv2_smem);   // [2][NZP][RY][RX]
    const int tid = threadIdx.x;
    const int rx = tid % RX, ry = tid / RX;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    int gx = (x0 - kHalo + rx) % nx;
    if (gx < 0) gx += nx;
    const int gy = y0 - kHalo + ry;
    const bool valid = gy >= 0 && gy < ny;
    const size_t plane = (size_t)nx * ny;
    const size_t col = valid ? (size_t)gy * nx + gx : 0;
    float c0 = 0.f, cE = 0.f, cW = 0.f, cN = 0.f, cS = 0.f;
    if (valid) {
        const float uL = a.u[col], uR = a.u[(size_t)gy * nx + (gx + 1 == nx ? 0 : gx + 1)];
        const float vS = a.v[col], vN = a.v[col + nx];
        const float uLp = fmaxf(uL, 0.f), uLm = fminf(uL, 0.f);
        const float uRp = fmaxf(uR, 0.f), uRm = fminf(uR, 0.f);
        const float vSp = fmaxf(vS, 0.f), vSm = fminf(vS, 0.f);
        const float vNp = fmaxf(vN, 0.f), vNm = fminf(vN, 0.f);
        c0 = (uLm - uRp) * a.rdx + (vSm - vNp) * a.rdy;
        if (!ADJ) {
            cE = -uRm * a.rdx;
            cW = uLp * a.rdx;
            cN = -vNm * a.rdy;
            cS = vSp * a.rdy;
        } else {
            cE = uRp * a.rdx;
            cW = -uLm * a.rdx;
            cN = vNp * a.rdy;
            cS = -vSm * a.rdy;
        }
    }
    const float2 C0 = make_float2(c0, c0), CE = make_float2(cE, cE), CW = make_float2(cW, cW);
    const float2 CN = make_float2(cN, cN), CS = make_float2(cS, cS);
    const size_t pb = (size_t)blockIdx.z * a.pstride;
    float2 c[NZP], w[NZP];
#pragma unroll
    for (int p = 0; p < NZP; ++p) {
        const int z0 = 2 * p, z1 = 2 * p + 1;
        c[p].x = (valid && z0 < nz) ? a.cin[pb + z0 * plane + col] : 0.f;
        c[p].y = (valid && z1 < nz) ? a.cin[pb + z1 * plane + col] : 0.f;
        w[p] = c[p];
    }
    float s0 = 0.f;
    if (!ADJ && valid && a.src) s0 = a.src[(size_t)blockIdx.z * a.sstride + col];
    float e0 = 0.f;
#pragma unroll
    for (int st = 0; st < 4; ++st) {
        float2 *S = S0 + (st & 1) * NZP * PL;
        // the stage input on the region of this stage grown by one column; rows beyond the
        // walls publish their zeros
        if (rx >= st && rx < RX - st && ry >= st && ry < RY - st) {
#pragma unroll
            for (int p = 0; p < NZP; ++p) S[p * PL + ry * RX + rx] = w[p];
        }
        if (ADJ && st == 3) e0 = w[0].x;
        __syncthreads();
        if (valid && rx > st && rx < RX - st - 1 && ry > st && ry < RY - st - 1) {
            const float al = (st == 0) ? 0.25f * a.h : (st == 1) ? a.h / 3.f : (st == 2) ? 0.5f * a.h : a.h;
            const float2 AL = make_float2(al, al);
            float below = 0.f;   // the stage input of level 2p - 1
#pragma unroll
            for (int p = 0; p < NZP; ++p) {
                const float2 wo = w[p];
                const float2 *Sp = S + p * PL + ry * RX + rx;
                float2 hor = __fmul2_rn(C0, wo);
                hor = __ffma2_rn(CE, Sp[1], hor);
                hor = __ffma2_rn(CW, Sp[-1], hor);
                hor = __ffma2_rn(CN, Sp[RX], hor);
                hor = __ffma2_rn(CS, Sp[-RX], hor);
                const float2 up = make_float2(wo.y, (p + 1 < NZP) ? w[p + 1].x : 0.f);
                const float2 dn = make_float2(below, wo.x);
                float2 k = __fmul2_rn(a.amp2[p], hor);
                k = __ffma2_rn(a.ku2[p], up, k);
                k = __ffma2_rn(a.kl2[p], dn, k);
                k = __ffma2_rn(a.nkd2[p], wo, k);
                if (!ADJ && p == 0) k.x += s0;
                w[p] = __ffma2_rn(AL, k, c[p]);
                below = wo.y;
            }
        }
    }
    const int ix = rx - kHalo, iy = ry - kHalo;
    if (valid && ix >= 0 && ix < TX && iy >= 0 && iy < TY && x0 + ix < nx) {
#pragma unroll
        for (int p = 0; p < NZP; ++p) {
            const int z0 = 2 * p, z1 = 2 * p + 1;
            if (z0 < nz) a.cout[pb + z0 * plane + col] = w[p].x;
            if (z1 < nz) a.cout[pb + z1 * plane + col] = w[p].y;
        }
        if (ADJ && a.ebar) a.ebar[(size_t)blockIdx.z * a.estride + col] += a.h * e0;
    }
}

template <typename R>
__global__ void obs_gather_kernel(const R *c, long long pstride, int o0, int no, const int *cell, const R *w,
                                  const R *rinv, R *r, long long rstride)
{
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= no) return;
    const int oo = o0 + o;
    const R *cp = c + (size_t)blockIdx.y * pstride;
    R acc = R(0);
#pragma unroll
    for (int q = 0; q < 8; ++q) acc += w[8 * oo + q] * cp[cell[8 * oo + q]];
    r[(size_t)blockIdx.y * rstride + oo] = rinv[oo] * acc;
}

__global__ void obs_innov_kernel(const double *c, int o0, int no, const int *cell, const double *w,
                                 const double *y, const double *rinv, double *d, double *jo)
{
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= no) return;
    const int oo = o0 + o;
    double acc = 0.0;
#pragma unroll
    for (int q = 0; q < 8; ++q) acc += w[8 * oo + q] * c[cell[8 * oo + q]];
    const double dd = acc - y[oo];
    d[oo] = dd;
    atomicAdd(jo, 0.5 * dd * dd * rinv[oo]);
}

template <typename R>
__global__ void obs_scatter_kernel(R *lam, long long pstride, int o0, int no, const int *cell, const R *w,
                                   const R *r, long long rstride)
{
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= no) return;
    const int oo = o0 + o;
    R *lp = lam + (size_t)blockIdx.y * pstride;
    const R rv = r[(size_t)blockIdx.y * rstride + oo];
#pragma unroll
    for (int q = 0; q < 8; ++q) atomicAdd(&lp[cell[8 * oo + q]], w[8 * oo + q] * rv);
}

// Batched row-major GEMM C_f = alpha A_f B_f (M x K times K x N); the batch
// index f maps to offsets (f / inner) * so + (f % inner) * si per operand.
template <typename R>
struct BGArgs {
    const R *A;
    const R *B;
    R *C;
    int M, N, K, inner;
    long long lda, ldb, ldc;
    long long aso, asi, bso, bsi, cso, csi;
    R alpha;
};

template <typename R>
__global__ void __launch_bounds__(256) bgemm_kernel(BGArgs<R> g)
{
    __shared__ R As[16][64 + 1];
    __shared__ R Bs[16][64 + 4];
    const int f = blockIdx.z;
    const R *A = g.A + (f / g.inner) * g.aso + (f % g.inner) * g.asi;
    const R *B = g.B + (f / g.inner) * g.bso + (f % g.inner) * g.bsi;
    R *C = g.C + (f / g.inner) * g.cso + (f % g.inner) * g.csi;
    const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    R acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = R(0);
    for (int k0 = 0; k0 < g.K; k0 += 16) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int idx = tid + 256 * i;
            const int mm = idx / 16, kk = idx % 16;
            As[kk][mm] = (m0 + mm < g.M && k0 + kk < g.K) ? A[(size_t)(m0 + mm) * g.lda + k0 + kk] : R(0);
            const int kb = idx / 64, nb = idx % 64;
            Bs[kb][nb] = (k0 + kb < g.K && n0 + nb < g.N) ? B[(size_t)(k0 + kb) * g.ldb + n0 + nb] : R(0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            R av[4], bv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) av[i] = As[kk][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] += av[i] * bv[j];
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int mm = m0 + ty * 4 + i;
        if (mm >= g.M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int nn = n0 + tx * 4 + j;
            if (nn < g.N) C[(size_t)mm * g.ldc + nn] = g.alpha * acc[i][j];
        }
    }
}

// out[j*ldo + i] = in[j*ldi + i] * s[i] (+ add[j*lda + i])
template <typename R>
__global__ void colscale_kernel(const R *in, long long ldi, const R *s, R *out, long long ldo, int n, int ncols)
{
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t total = (size_t)n * ncols;
    if (t >= total) return;
    const int j = (int)(t / n), i = (int)(t % n);
    out[(size_t)j * ldo + i] = in[(size_t)j * ldi + i] * s[i];
}

template <typename R>
__global__ void coladd_kernel(const R *in, long long ldi, R *out, long long ldo, int n, int ncols)
{
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t total = (size_t)n * ncols;
    if (t >= total) return;
    const int j = (int)(t / n), i = (int)(t % n);
    out[(size_t)j * ldo + i] += in[(size_t)j * ldi + i];
}

__global__ void emis_scale_kernel(const double *Eb, const double *x, double rdz, int n, double *Es64, float *Es32)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double e = Eb[i] * exp(x[i]) * rdz;
    Es64[i] = e;
    if (Es32) Es32[i] = (float)e;
}

inline unsigned blocks_for(size_t n, int t) { return (unsigned)((n + t - 1) / t); }

template <typename R>
struct Tab;
template <>
struct Tab<float> {
    static const float *u(const AdvDev &m) { return m.u32; }
    static const float *v(const AdvDev &m) { return m.v32; }
    static const float *amp(const AdvDev &m) { return m.amp32; }
    static const float *kz(const AdvDev &m) { return m.kz32; }
    static const float *w(const AdvDev &m) { return m.w32; }
    static const float *rinv(const AdvDev &m) { return m.rinv32; }
    static const float *Sx(const AdvDev &m) { return m.Sx32; }
    static const float *Sy(const AdvDev &m) { return m.Sy32; }
    static const float *Es(const AdvDev &m) { return m.Es32; }
};
template <>
struct Tab<double> {
    static const double *u(const AdvDev &m) { return m.u64; }
    static const double *v(const AdvDev &m) { return m.v64; }
    static const double *amp(const AdvDev &m) { return m.amp64; }
    static const double *kz(const AdvDev &m) { return m.kz64; }
    static const double *w(const AdvDev &m) { return m.w64; }
    static const double *rinv(const AdvDev &m) { return m.rinv64; }
    static const double *Sx(const AdvDev &m) { return m.Sx64; }
    static const double *Sy(const AdvDev &m) { return m.Sy64; }
    static const double *Es(const AdvDev &m) { return m.Es64; }
};

// Tile shape per precision: FP32 keeps 3 x NZ floats per thread with 480
// threads; FP64 needs twice the registers per level, so its tiles are smaller.
template <typename R>
struct TileShape;
template <>
struct TileShape<float> {
    static constexpr int TX = 32, TY = 4;
};
template <>
struct TileShape<double> {
    static constexpr int TX = 16, TY = 2;
};

template <typename R, int NZ, bool ADJ>
cudaError_t step_nz(const StepArgs<R> &a, int P, cudaStream_t s)
{
    constexpr int TX = TileShape<R>::TX, TY = TileShape<R>::TY;
    constexpr int RX = TX + 2 * kHalo, RY = TY + 2 * kHalo;
    const size_t smem = sizeof(R) * 2 * (size_t)NZ * RX * RY;
    auto kern = adv_step_kernel<R, NZ, TX, TY, ADJ>;
    static bool attr_done = false;
    if (!attr_done) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_done = true;
    }
    dim3 grid((a.nx + TX - 1) / TX, (a.ny + TY - 1) / TY, P);
    kern<<<grid, RX * RY, smem, s>>>(a);
    count_launch();
    return cudaGetLastError();
}

template <int NZP, int TX, int TY, bool ADJ>
cudaError_t step_f2_nz(const StepArgsF2 &a, int P, cudaStream_t s)
{
    constexpr int RX = TX + 2 * kHalo, RY = TY + 2 * kHalo;
    const size_t smem = sizeof(float2) * 2 * (size_t)NZP * RX * RY;
    auto kern = adv_step_f2_kernel<NZP, TX, TY, ADJ>;
    static bool attr_done = false;
    if (!attr_done) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_done = true;
    }
    dim3 grid((a.nx + TX - 1) / TX, (a.ny + TY - 1) / TY, P);
    kern<<<grid, RX * RY, smem, s>>>(a);
    count_launch();
    return cudaGetLastError();
}

// FP32 steps: the packed nested kernel (levels in pairs; 32 x 8 tiles of 640 threads up to 30
// levels, 24 x 8 tiles of 512 threads with 128 registers for 32 levels; measured on the
// 30-level grid, 32 x 8 tiles at 96 registers beat 24 x 8 at 128, and beat a persistent form
// that prefetched the next tile's input into the free plane, whose loop spilled registers)
cudaError_t step_f32(const AdvDev &m, const float *cin, float *cout, int P, const float *src, long long sstride,
                     float *ebar, long long estride, bool adj, cudaStream_t s)
{
    StepArgsF2 a;
    const int nzp = m.nz <= 8 ? 4 : m.nz <= 16 ? 8 : m.nz <= 30 ? 15 : 16;
    for (int p = 0; p < 16; ++p) {
        const int z0 = 2 * p, z1 = 2 * p + 1;
        auto kz = [&](int l) { return (l > 0 && l < m.nz) ? (float)(m.kz_h[l] / (m.dz * m.dz)) : 0.f; };
        a.amp2[p] = make_float2(z0 < m.nz ? (float)m.amp_h[z0] : 0.f, z1 < m.nz ? (float)m.amp_h[z1] : 0.f);
        a.ku2[p] = make_float2(kz(z0 + 1), kz(z1 + 1));
        a.kl2[p] = make_float2(kz(z0), kz(z1));
        a.nkd2[p] = make_float2(-(a.ku2[p].x + a.kl2[p].x), -(a.ku2[p].y + a.kl2[p].y));
    }
    a.cin = cin;
    a.cout = cout;
    a.pstride = m.ncells;
    a.src = src;
    a.sstride = sstride;
    a.ebar = ebar;
    a.estride = estride;
    a.u = m.u32;
    a.v = m.v32;
    a.nx = m.nx;
    a.ny = m.ny;
    a.nz = m.nz;
    a.h = (float)m.dt;
    a.rdx = (float)(1.0 / m.dx);
    a.rdy = (float)(1.0 / m.dy);
    if (nzp == 4) return adj ? step_f2_nz<4, 32, 8, true>(a, P, s) : step_f2_nz<4, 32, 8, false>(a, P, s);
    if (nzp == 8) return adj ? step_f2_nz<8, 32, 8, true>(a, P, s) : step_f2_nz<8, 32, 8, false>(a, P, s);
    if (nzp == 15) return adj ? step_f2_nz<15, 32, 8, true>(a, P, s) : step_f2_nz<15, 32, 8, false>(a, P, s);
    return adj ? step_f2_nz<16, 24, 8, true>(a, P, s) : step_f2_nz<16, 24, 8, false>(a, P, s);
}

template <typename R>
cudaError_t step(const AdvDev &m, const R *cin, R *cout, int P, const R *src, long long sstride, R *ebar,
                 long long estride, bool adj, cudaStream_t s)
{
    if constexpr (sizeof(R) == sizeof(float)) return step_f32(m, cin, cout, P, src, sstride, ebar, estride, adj, s);
    StepArgs<R> a;
    a.cin = cin;
    a.cout = cout;
    a.pstride = m.ncells;
    a.src = src;
    a.sstride = sstride;
    a.ebar = ebar;
    a.estride = estride;
    a.u = Tab<R>::u(m);
    a.v = Tab<R>::v(m);
    for (int l = 0; l < kMaxNZ; ++l) a.amp[l] = l < m.nz ? (R)m.amp_h[l] : R(0);
    for (int l = 0; l <= kMaxNZ; ++l)
        a.kzs[l] = (l > 0 && l < m.nz) ? (R)(m.kz_h[l] / (m.dz * m.dz)) : R(0);
    a.nx = m.nx;
    a.ny = m.ny;
    a.nz = m.nz;
    a.h = (R)m.dt;
    a.rdx = (R)(1.0 / m.dx);
    a.rdy = (R)(1.0 / m.dy);
    if (m.nz <= 8) return adj ? step_nz<R, 8, true>(a, P, s) : step_nz<R, 8, false>(a, P, s);
    if (m.nz <= 16) return adj ? step_nz<R, 16, true>(a, P, s) : step_nz<R, 16, false>(a, P, s);
    return adj ? step_nz<R, 32, true>(a, P, s) : step_nz<R, 32, false>(a, P, s);
}

template <typename R>
cudaError_t gather(const AdvDev &m, const R *c, int P, int t, R *r, long long rstride, cudaStream_t s)
{
    const int o0 = m.optr_h[t], no = m.optr_h[t + 1] - o0;
    if (no <= 0) return cudaSuccess;
    dim3 grid(blocks_for(no, 128), P);
    obs_gather_kernel<R><<<grid, 128, 0, s>>>(c, m.ncells, o0, no, m.cell, Tab<R>::w(m), Tab<R>::rinv(m), r, rstride);
    count_launch();
    return cudaGetLastError();
}

template <typename R>
cudaError_t scatter(const AdvDev &m, R *lam, int P, int t, const R *r, long long rstride, cudaStream_t s)
{
    const int o0 = m.optr_h[t], no = m.optr_h[t + 1] - o0;
    if (no <= 0) return cudaSuccess;
    dim3 grid(blocks_for(no, 128), P);
    obs_scatter_kernel<R><<<grid, 128, 0, s>>>(lam, m.ncells, o0, no, m.cell, Tab<R>::w(m), r, rstride);
    count_launch();
    return cudaGetLastError();
}

template <typename R>
cudaError_t bgemm(const BGArgs<R> &g, int batch, cudaStream_t s)
{
    dim3 grid((g.N + 63) / 64, (g.M + 63) / 64, batch);
    bgemm_kernel<R><<<grid, 256, 0, s>>>(g);
    count_launch();
    return cudaGetLastError();
}

// out (ncols columns at ldo) = sigma_b (S_y kron S_x) in (ncols columns at ldi),
// per emission block; tmp holds ncols * n reals.  S_x, S_y are symmetric, so
// this is also L^T.
template <typename R>
cudaError_t sep_apply(const AdvDev &m, const R *in, long long ldi, R *out, long long ldo, int ncols, R *tmp,
                      cudaStream_t s)
{
    const long long nyx = (long long)m.ny * m.nx;
    const int batch = ncols * m.nb;
    // tmp_f = F_f S_x   (ny x nx) (nx x nx)
    BGArgs<R> g1;
    g1.A = in;
    g1.B = Tab<R>::Sx(m);
    g1.C = tmp;
    g1.M = m.ny;
    g1.N = m.nx;
    g1.K = m.nx;
    g1.inner = m.nb;
    g1.lda = m.nx;
    g1.ldb = m.nx;
    g1.ldc = m.nx;
    g1.aso = ldi;
    g1.asi = nyx;
    g1.bso = 0;
    g1.bsi = 0;
    g1.cso = (long long)m.nb * nyx;
    g1.csi = nyx;
    g1.alpha = R(1);
    cudaError_t e = bgemm(g1, batch, s);
    if (e != cudaSuccess) return e;
    // out_f = sigma_b S_y tmp_f   (ny x ny) (ny x nx)
    BGArgs<R> g2;
    g2.A = Tab<R>::Sy(m);
    g2.B = tmp;
    g2.C = out;
    g2.M = m.ny;
    g2.N = m.nx;
    g2.K = m.ny;
    g2.inner = m.nb;
    g2.lda = m.ny;
    g2.ldb = m.nx;
    g2.ldc = m.nx;
    g2.aso = 0;
    g2.asi = 0;
    g2.bso = (long long)m.nb * nyx;
    g2.bsi = nyx;
    g2.cso = ldo;
    g2.csi = nyx;
    g2.alpha = (R)m.sigma_b;
    return bgemm(g2, batch, s);
}

template <typename R>
cudaError_t colscale(const R *in, long long ldi, const R *sc, R *out, long long ldo, int n, int ncols, cudaStream_t s)
{
    const size_t total = (size_t)n * ncols;
    if (!total) return cudaSuccess;
    colscale_kernel<R><<<blocks_for(total, 256), 256, 0, s>>>(in, ldi, sc, out, ldo, n, ncols);
    count_launch();
    return cudaGetLastError();
}

template <typename R>
cudaError_t hvp_batch(const AdvDev &m, const R *W, R *Y, long long ld, int P, int add_identity, R *r, cudaStream_t s)
{
    cudaError_t e;
    const long long n = m.n, nyx = (long long)m.ny * m.nx;
    R *cA = (R *)m.cA, *cB = (R *)m.cB, *src = (R *)m.src, *ebar = (R *)m.ebar, *tmp = (R *)m.tmp;
    const size_t cells = (size_t)P * m.ncells;
#define ADV_TRY(x)                          \
    do {                                    \
        if ((e = (x)) != cudaSuccess) return e; \
    } while (0)
    // source perturbation: E / dz * (L w)
    ADV_TRY(sep_apply<R>(m, W, ld, src, n, P, tmp, s));
    ADV_TRY(colscale<R>(src, n, Tab<R>::Es(m), src, n, (int)n, P, s));
    // tangent-linear window, residuals r = R^-1 H dc at the observation steps
    ADV_TRY(cudaMemsetAsync(cA, 0, cells * sizeof(R), s));
    for (int t = 0; t < m.T; ++t) {
        const int b = (int)(((long long)t * m.nb) / m.T);
        ADV_TRY(step<R>(m, cA, cB, P, src + b * nyx, n, nullptr, 0, false, s));
        R *sw = cA;
        cA = cB;
        cB = sw;
        ADV_TRY(gather<R>(m, cA, P, t + 1, r, m.p, s));
    }
    // adjoint window
    ADV_TRY(cudaMemsetAsync(cA, 0, cells * sizeof(R), s));
    ADV_TRY(cudaMemsetAsync(ebar, 0, (size_t)P * n * sizeof(R), s));
    for (int t = m.T - 1; t >= 0; --t) {
        ADV_TRY(scatter<R>(m, cA, P, t + 1, r, m.p, s));
        const int b = (int)(((long long)t * m.nb) / m.T);
        ADV_TRY(step<R>(m, cA, cB, P, nullptr, 0, ebar + b * nyx, n, true, s));
        R *sw = cA;
        cA = cB;
        cB = sw;
    }
    // Y = L^T (E / dz * ebar) (+ W)
    ADV_TRY(colscale<R>(ebar, n, Tab<R>::Es(m), ebar, n, (int)n, P, s));
    ADV_TRY(sep_apply<R>(m, ebar, n, Y, ld, P, tmp, s));
    if (add_identity) {
        const size_t total = (size_t)n * P;
        coladd_kernel<R><<<blocks_for(total, 256), 256, 0, s>>>(W, ld, Y, ld, (int)n, P);
        count_launch();
        ADV_TRY(cudaGetLastError());
    }
#undef ADV_TRY
    return cudaSuccess;
}

// The two halves of a product on P columns, for the observation-space dual of Algorithm 4:
// tangent linear r = R^-1 H' L w (ld ldw, r with stride p) and adjoint z = L^T H'^T f from an
// observation-space forcing f (stride p; z at ld ldz).
template <typename R>
cudaError_t tl_batch(const AdvDev &m, const R *W, long long ldw, int P, R *r, cudaStream_t s)
{
    cudaError_t e;
    const long long n = m.n, nyx = (long long)m.ny * m.nx;
    R *cA = (R *)m.cA, *cB = (R *)m.cB, *src = (R *)m.src, *tmp = (R *)m.tmp;
    const size_t cells = (size_t)P * m.ncells;
    if ((e = sep_apply<R>(m, W, ldw, src, n, P, tmp, s)) != cudaSuccess) return e;
    if ((e = colscale<R>(src, n, Tab<R>::Es(m), src, n, (int)n, P, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(cA, 0, cells * sizeof(R), s)) != cudaSuccess) return e;
    for (int t = 0; t < m.T; ++t) {
        const int b = (int)(((long long)t * m.nb) / m.T);
        if ((e = step<R>(m, cA, cB, P, src + b * nyx, n, nullptr, 0, false, s)) != cudaSuccess) return e;
        R *sw = cA;
        cA = cB;
        cB = sw;
        if ((e = gather<R>(m, cA, P, t + 1, r, m.p, s)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <typename R>
cudaError_t ad_batch(const AdvDev &m, const R *f, int P, R *Z, long long ldz, cudaStream_t s)
{
    cudaError_t e;
    const long long n = m.n, nyx = (long long)m.ny * m.nx;
    R *cA = (R *)m.cA, *cB = (R *)m.cB, *ebar = (R *)m.ebar, *tmp = (R *)m.tmp;
    const size_t cells = (size_t)P * m.ncells;
    if ((e = cudaMemsetAsync(cA, 0, cells * sizeof(R), s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(ebar, 0, (size_t)P * n * sizeof(R), s)) != cudaSuccess) return e;
    for (int t = m.T - 1; t >= 0; --t) {
        if ((e = scatter<R>(m, cA, P, t + 1, f, m.p, s)) != cudaSuccess) return e;
        const int b = (int)(((long long)t * m.nb) / m.T);
        if ((e = step<R>(m, cA, cB, P, nullptr, 0, ebar + b * nyx, n, true, s)) != cudaSuccess) return e;
        R *sw = cA;
        cA = cB;
        cB = sw;
    }
    if ((e = colscale<R>(ebar, n, Tab<R>::Es(m), ebar, n, (int)n, P, s)) != cudaSuccess) return e;
    return sep_apply<R>(m, ebar, n, Z, ldz, P, tmp, s);
}

}  // namespace

cudaError_t adv_tl(const AdvDev &m, const double *W, int64_t ld, int ncols, double *r, cudaStream_t s)
{
    for (int c0 = 0; c0 < ncols; c0 += m.Pws64) {
        const int P = ncols - c0 < m.Pws64 ? ncols - c0 : m.Pws64;
        cudaError_t e = tl_batch<double>(m, W + (size_t)c0 * ld, ld, P, r + (size_t)c0 * m.p, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t adv_ad(const AdvDev &m, const double *f, int ncols, double *Z, int64_t ld, cudaStream_t s)
{
    for (int c0 = 0; c0 < ncols; c0 += m.Pws64) {
        const int P = ncols - c0 < m.Pws64 ? ncols - c0 : m.Pws64;
        cudaError_t e = ad_batch<double>(m, f + (size_t)c0 * m.p, P, Z + (size_t)c0 * ld, ld, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t adv_ad_obs(const AdvDev &m, const double *f, double *z, cudaStream_t s)
{
    cudaError_t e;
    const long long n = m.n, nyx = (long long)m.ny * m.nx;
    double *cA = m.c64A, *cB = m.c64B;
    if ((e = cudaMemsetAsync(cA, 0, (size_t)m.ncells * sizeof(double), s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(m.ebar64, 0, (size_t)n * sizeof(double), s)) != cudaSuccess) return e;
    for (int t = m.T - 1; t >= 0; --t) {
        if ((e = scatter<double>(m, cA, 1, t + 1, f, m.p, s)) != cudaSuccess) return e;
        const int bk = (int)(((long long)t * m.nb) / m.T);
        if ((e = step<double>(m, cA, cB, 1, nullptr, 0, m.ebar64 + bk * nyx, n, true, s)) != cudaSuccess) return e;
        double *sw = cA;
        cA = cB;
        cB = sw;
    }
    if ((e = colscale<double>(m.ebar64, n, m.Es64, m.ebar64, n, (int)n, 1, s)) != cudaSuccess) return e;
    return sep_apply<double>(m, m.ebar64, n, z, n, 1, m.tmp64, s);
}

cudaError_t adv_hvp(const AdvDev &m, bool fp64, const void *W, void *Y, int64_t ld, int ncols, int add_identity,
                    void *r, cudaStream_t s)
{
    for (int c0 = 0; c0 < ncols; c0 += m.Pmax) {
        const int P = ncols - c0 < m.Pmax ? ncols - c0 : m.Pmax;
        cudaError_t e;
        if (fp64)
            e = hvp_batch<double>(m, (const double *)W + (size_t)c0 * ld, (double *)Y + (size_t)c0 * ld, ld, P,
                                  add_identity, (double *)r, s);
        else
            e = hvp_batch<float>(m, (const float *)W + (size_t)c0 * ld, (float *)Y + (size_t)c0 * ld, ld, P,
                                 add_identity, (float *)r, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t adv_outer(const AdvDev &m, const double *x, double *d, double *jo, double *rd, double *b, cudaStream_t s)
{
    cudaError_t e;
    const long long n = m.n, nyx = (long long)m.ny * m.nx;
    emis_scale_kernel<<<blocks_for(n, 256), 256, 0, s>>>(m.Eb, x, 1.0 / m.dz, (int)n, m.Es64, m.Es32);
    count_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    double *cA = m.c64A, *cB = m.c64B;
    // nonlinear window (the transport is linear in the tracer; the source is E(x) / dz)
    if ((e = cudaMemsetAsync(cA, 0, (size_t)m.ncells * sizeof(double), s)) != cudaSuccess) return e;
    for (int t = 0; t < m.T; ++t) {
        const int bk = (int)(((long long)t * m.nb) / m.T);
        if ((e = step<double>(m, cA, cB, 1, m.Es64 + bk * nyx, 0, nullptr, 0, false, s)) != cudaSuccess) return e;
        double *sw = cA;
        cA = cB;
        cB = sw;
        const int o0 = m.optr_h[t + 1], no = m.optr_h[t + 2] - o0;
        if (no > 0) {
            obs_innov_kernel<<<blocks_for(no, 128), 128, 0, s>>>(cA, o0, no, m.cell, m.w64, m.y, m.rinv64, d, jo);
            count_launch();
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
    }
    // gradient b = L^T (E / dz * ebar), ebar the source adjoint of R^-1 d
    if (m.p > 0) {
        if ((e = mul(m.p, d, m.rinv64, rd, s)) != cudaSuccess) return e;
    }
    if ((e = cudaMemsetAsync(cA, 0, (size_t)m.ncells * sizeof(double), s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(m.ebar64, 0, (size_t)n * sizeof(double), s)) != cudaSuccess) return e;
    for (int t = m.T - 1; t >= 0; --t) {
        if ((e = scatter<double>(m, cA, 1, t + 1, rd, m.p, s)) != cudaSuccess) return e;
        const int bk = (int)(((long long)t * m.nb) / m.T);
        if ((e = step<double>(m, cA, cB, 1, nullptr, 0, m.ebar64 + bk * nyx, n, true, s)) != cudaSuccess) return e;
        double *sw = cA;
        cA = cB;
        cB = sw;
    }
    if ((e = colscale<double>(m.ebar64, n, m.Es64, m.ebar64, n, (int)n, 1, s)) != cudaSuccess) return e;
    return sep_apply<double>(m, m.ebar64, n, b, n, 1, m.tmp64, s);
}

cudaError_t adv_tl_obs(const AdvDev &m, const double *w, double *r, cudaStream_t s)
{
    cudaError_t e;
    const long long n = m.n, nyx = (long long)m.ny * m.nx;
    double *cA = m.c64A, *cB = m.c64B, *src = m.ebar64;
    // source perturbation E / dz * (L w), then the tangent-linear window from zero
    if ((e = sep_apply<double>(m, w, n, src, n, 1, m.tmp64, s)) != cudaSuccess) return e;
    if ((e = colscale<double>(src, n, m.Es64, src, n, (int)n, 1, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(cA, 0, (size_t)m.ncells * sizeof(double), s)) != cudaSuccess) return e;
    for (int t = 0; t < m.T; ++t) {
        const int bk = (int)(((long long)t * m.nb) / m.T);
        if ((e = step<double>(m, cA, cB, 1, src + bk * nyx, n, nullptr, 0, false, s)) != cudaSuccess) return e;
        double *sw = cA;
        cA = cB;
        cB = sw;
        if ((e = gather<double>(m, cA, 1, t + 1, r, m.p, s)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t adv_bsqrt(const AdvDev &m, const double *in, double *out, int ncols, cudaStream_t s)
{
    for (int c0 = 0; c0 < ncols; c0 += m.Pmax64) {
        const int P = ncols - c0 < m.Pmax64 ? ncols - c0 : m.Pmax64;
        cudaError_t e = sep_apply<double>(m, in + (size_t)c0 * m.n, m.n, out + (size_t)c0 * m.n, m.n, P, m.tmp64, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// One column of the tracer forecast from x (FP64): the tracer field after
// steps steps, for building synthetic truths and tests.
cudaError_t adv_forecast(const AdvDev &m, const double *x, int steps, double *c_out, cudaStream_t s)
{
    cudaError_t e;
    const long long n = m.n, nyx = (long long)m.ny * m.nx;
    emis_scale_kernel<<<blocks_for(n, 256), 256, 0, s>>>(m.Eb, x, 1.0 / m.dz, (int)n, m.Es64, m.Es32);
    count_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    double *cA = m.c64A, *cB = m.c64B;
    if ((e = cudaMemsetAsync(cA, 0, (size_t)m.ncells * sizeof(double), s)) != cudaSuccess) return e;
    for (int t = 0; t < steps; ++t) {
        const int bk = (int)(((long long)t * m.nb) / m.T);
        if ((e = step<double>(m, cA, cB, 1, m.Es64 + bk * nyx, 0, nullptr, 0, false, s)) != cudaSuccess) return e;
        double *sw = cA;
        cA = cB;
        cB = sw;
    }
    return cudaMemcpyAsync(c_out, cA, (size_t)m.ncells * sizeof(double), cudaMemcpyDeviceToDevice, s);
}

}  // namespace riot
