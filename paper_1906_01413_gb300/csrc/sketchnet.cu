// Learned sketch proposal: a periodic 1-D conv-net maps snapshots of a
// Lorenz-96 background trajectory to m proposed sketch directions.  Forward
// (FP32, or BF16-rounded weights and activations with FP32 accumulation for
// inference), backward, the subspace loss and Adam, all as kernels here; the
// Gaussian sketch of Algorithm 3 stays the fallback (riot_rsvd_proposal).
//
// Layout: activations [B][C][n] (FP32), parameters one flat FP32 vector, per
// layer W[C_out][C_in][K] then b[C_out].  conv(x)[o][i] = b[o] +
// sum_c sum_d W[o][c][d] x[c][(i + d - h) mod n], h = K / 2.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>

#include "internal.h"

namespace riot {

namespace {

constexpr int kOutPerThread = 8;

__device__ __forceinline__ float bf16r(float v) { return __bfloat162float(__float2bfloat16(v)); }

// out[b][o][i] = act(b[o] + sum_c sum_d W[o][c][d] in[b][c][(i + d - h) mod n])
template <bool TANH, bool BF16>
__global__ void __launch_bounds__(128) conv_fwd_kernel(const float *in, int ci, const float *W, const float *bias,
                                                       float *out, int co, int n, int K)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int o0 = blockIdx.y * kOutPerThread;
    const int b = blockIdx.z;
    if (i >= n) return;
    const int h = K / 2;
    float acc[kOutPerThread];
#pragma unroll
    for (int q = 0; q < kOutPerThread; ++q) {
        const int o = o0 + q;
        acc[q] = (o < co) ? (BF16 ? bf16r(bias[o]) : bias[o]) : 0.f;
    }
    const float *xb = in + (size_t)b * ci * n;
    for (int c = 0; c < ci; ++c) {
        for (int d = 0; d < K; ++d) {
            int j = i + d - h;
            j += (j < 0) ? n : 0;
            j -= (j >= n) ? n : 0;
            float x = xb[(size_t)c * n + j];
            if (BF16) x = bf16r(x);
#pragma unroll
            for (int q = 0; q < kOutPerThread; ++q) {
                const int o = o0 + q;
                if (o < co) {
                    float w = W[((size_t)o * ci + c) * K + d];
                    if (BF16) w = bf16r(w);
                    acc[q] = fmaf(w, x, acc[q]);
                }
            }
        }
    }
    float *ob = out + (size_t)b * co * n;
#pragma unroll
    for (int q = 0; q < kOutPerThread; ++q) {
        const int o = o0 + q;
        if (o < co) {
            float v = TANH ? tanhf(acc[q]) : acc[q];
            if (BF16) v = bf16r(v);
            ob[(size_t)o * n + i] = v;
        }
    }
}

// gin[b][c][j] = (sum_o sum_d W[o][c][d] gout[b][o][(j - d + h) mod n]) * (1 - act[b][c][j]^2)
__global__ void __launch_bounds__(128) conv_bwd_data_kernel(const float *gout, int co, const float *W,
                                                            const float *act, float *gin, int ci, int n, int K)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int c0 = blockIdx.y * kOutPerThread;
    const int b = blockIdx.z;
    if (j >= n) return;
    const int h = K / 2;
    float acc[kOutPerThread];
#pragma unroll
    for (int q = 0; q < kOutPerThread; ++q) acc[q] = 0.f;
    const float *gb = gout + (size_t)b * co * n;
    for (int o = 0; o < co; ++o) {
        for (int d = 0; d < K; ++d) {
            int i = j - d + h;
            i += (i < 0) ? n : 0;
            i -= (i >= n) ? n : 0;
            const float g = gb[(size_t)o * n + i];
#pragma unroll
            for (int q = 0; q < kOutPerThread; ++q) {
                const int c = c0 + q;
                if (c < ci) acc[q] = fmaf(W[((size_t)o * ci + c) * K + d], g, acc[q]);
            }
        }
    }
#pragma unroll
    for (int q = 0; q < kOutPerThread; ++q) {
        const int c = c0 + q;
        if (c < ci) {
            const size_t idx = ((size_t)b * ci + c) * n + j;
            const float a = act[idx];
            gin[idx] = acc[q] * (1.f - a * a);
        }
    }
}

// gW[o][c][d] = sum_b sum_i gout[b][o][i] in[b][c][(i + d - h) mod n]; gb[o] (c == 0 blocks)
__global__ void __launch_bounds__(256) conv_bwd_weight_kernel(const float *gout, int co, const float *in, int ci,
                                                              int n, int K, int B, float *gW, float *gbias)
{
    const int o = blockIdx.x / ci, c = blockIdx.x % ci;
    const int h = K / 2;
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    double accb = 0.0;
    for (int b = 0; b < B; ++b) {
        const float *g = gout + ((size_t)b * co + o) * n;
        const float *x = in + ((size_t)b * ci + c) * n;
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const float gv = g[i];
            for (int d = 0; d < K && d < 8; ++d) {
                int j = i + d - h;
                j += (j < 0) ? n : 0;
                j -= (j >= n) ? n : 0;
                acc[d] += (double)gv * (double)x[j];
            }
            accb += gv;
        }
    }
    __shared__ double red[8][256];
    __shared__ double redb[256];
    for (int d = 0; d < 8; ++d) red[d][threadIdx.x] = acc[d];
    redb[threadIdx.x] = accb;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            for (int d = 0; d < 8; ++d) red[d][threadIdx.x] += red[d][threadIdx.x + s];
            redb[threadIdx.x] += redb[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        for (int d = 0; d < K && d < 8; ++d) gW[((size_t)o * ci + c) * K + d] = (float)red[d][0];
        if (c == 0) gbias[o] = (float)redb[0];
    }
}

// out[0] += sum x^2 (double accumulation), for the loss normalisers
__global__ void sumsq_kernel(const float *x, size_t n, double *out)
{
    double s = 0.0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const double v = x[i];
        s += v * v;
    }
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0 && s != 0.0) atomicAdd(out, s);
}

// Per-window loss scalars from sc = [a = ||R||^2, b = ||X||^2, ||E||^2, tr(E S)] and
// the window's Gram S (m x m, scaled in place to S / s and E = S - I written to E).
__global__ void gram_to_e_kernel(const float *G, int m, const double *sc, float *E, double *esc)
{
    const double s = sc[1] / m;
    double e2 = 0.0, tr = 0.0;
    for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
        const int i = t % m, j = t / m;
        const double S = (double)G[t] / s;
        const double e = S - (i == j ? 1.0 : 0.0);
        E[t] = (float)e;
        e2 += e * e;
        tr += e * S;
    }
    for (int off = 16; off > 0; off >>= 1) {
        e2 += __shfl_xor_sync(0xffffffffu, e2, off);
        tr += __shfl_xor_sync(0xffffffffu, tr, off);
    }
    __shared__ double r1[32], r2[32];
    if ((threadIdx.x & 31) == 0) {
        r1[threadIdx.x / 32] = e2;
        r2[threadIdx.x / 32] = tr;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0, c = 0;
        for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) {
            a += r1[w];
            c += r2[w];
        }
        esc[0] = a;
        esc[1] = c;
    }
}

// gX = c1 R + c2 X + c3 (X E), with the window's scalars; loss += (L1 + mu L2) / B
__global__ void loss_combine_kernel(const float *R, const float *X, const float *XE, size_t nm, int m, double mu,
                                    int B, const double *sc, const double *esc, float *gX, double *loss)
{
    const double b = sc[1], L1 = sc[0] / b, s = b / m;
    const double L2 = esc[0] / ((double)m * m), trES = esc[1];
    const double k2 = 4.0 / ((double)m * m * s);
    const double c1 = 2.0 / b / B, c2 = (-2.0 * L1 / b - mu * k2 * trES / m) / B, c3 = mu * k2 / B;
    for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < nm; t += (size_t)gridDim.x * blockDim.x)
        gX[t] = (float)(c1 * R[t] + c2 * X[t] + c3 * XE[t]);
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(loss, (L1 + mu * L2) / B);
}

__global__ void adam_kernel(float *p, const float *g, float *m, float *v, int64_t n, float lr, float b1, float b2,
                            float eps, float c1, float c2)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// x[c][i] = traj[floor(c T / C)][i] (FP32), and the mean / sum of squares into st[0..1]
__global__ void snapshot_kernel(const double *traj, int T, int64_t n, int C, float *x, double *st)
{
    double s = 0.0, s2 = 0.0;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n * C; t += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(t / n);
        const int64_t i = t - (int64_t)c * n;
        const int step = (int)(((int64_t)c * T) / C);
        const double v = traj[(int64_t)step * n + i];
        x[t] = (float)v;
        s += v;
        s2 += v * v;
    }
    for (int off = 16; off > 0; off >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, off);
        s2 += __shfl_xor_sync(0xffffffffu, s2, off);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&st[0], s);
        atomicAdd(&st[1], s2);
    }
}

__global__ void standardise_kernel(const double *traj, int T, int64_t n, int C, float *x, const double *st)
{
    const double N = (double)n * C;
    const double mean = st[0] / N;
    const double var = st[1] / N - mean * mean;
    const double inv = var > 0.0 ? 1.0 / sqrt(var) : 1.0;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n * C; t += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(t / n);
        const int64_t i = t - (int64_t)c * n;
        const int step = (int)(((int64_t)c * T) / C);
        x[t] = (float)((traj[(int64_t)step * n + i] - mean) * inv);
    }
}

inline unsigned blocks_for(size_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

// ---------------------------------------------------------------------------
int64_t SketchNet::num_params() const
{
    int64_t tot = 0;
    for (int l = 0; l < depth; ++l) tot += (int64_t)chan[l + 1] * chan[l] * K + chan[l + 1];
    return tot;
}

int64_t SketchNet::w_offset(int l) const
{
    int64_t o = 0;
    for (int j = 0; j < l; ++j) o += (int64_t)chan[j + 1] * chan[j] * K + chan[j + 1];
    return o;
}

cudaError_t sketchnet_forward(const SketchNet &net, const float *params, const float *x, int n, int B, float *Z,
                              bool bf16, float *acts, cudaStream_t s)
{
    // acts: (depth - 1) hidden layers of B * width * n floats, or nullptr to use ping-pong scratch
    const float *in = x;
    for (int l = 0; l < net.depth; ++l) {
        const int ci = net.chan[l], co = net.chan[l + 1];
        const float *W = params + net.w_offset(l);
        const float *bias = W + (size_t)co * ci * net.K;
        float *out = (l == net.depth - 1) ? Z : acts + (size_t)l * B * net.width * n;
        dim3 grid(blocks_for(n, 128), (co + kOutPerThread - 1) / kOutPerThread, B);
        const bool tanh_act = l < net.depth - 1;
        count_launch();
        if (tanh_act && bf16) conv_fwd_kernel<true, true><<<grid, 128, 0, s>>>(in, ci, W, bias, out, co, n, net.K);
        else if (tanh_act) conv_fwd_kernel<true, false><<<grid, 128, 0, s>>>(in, ci, W, bias, out, co, n, net.K);
        else if (bf16) conv_fwd_kernel<false, true><<<grid, 128, 0, s>>>(in, ci, W, bias, out, co, n, net.K);
        else conv_fwd_kernel<false, false><<<grid, 128, 0, s>>>(in, ci, W, bias, out, co, n, net.K);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        in = out;
    }
    return cudaSuccess;
}

cudaError_t sketchnet_loss_grad(const SketchNet &net, const float *params, const float *x, const float *U, int r,
                                int n, int B, double mu, float *grad, double *loss_dev, SketchWork &w,
                                cudaStream_t s)
{
    const int m = net.m;
    cudaError_t e;
    if ((e = sketchnet_forward(net, params, x, n, B, w.Z, false, w.acts, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(loss_dev, 0, sizeof(double), s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(w.sc, 0, sizeof(double) * 4 * B, s)) != cudaSuccess) return e;
    const size_t nm = (size_t)n * m;
    for (int b = 0; b < B; ++b) {
        const float *X = w.Z + (size_t)b * nm;          // n x m column-major: column j = direction j
        const float *Ub = U + (size_t)b * n * r;
        float *gX = w.gZ + (size_t)b * nm;
        double *sc = w.sc + 4 * b;
        // R = X - U (U^T X)
        if ((e = cudaMemcpyAsync(w.R, X, sizeof(float) * nm, cudaMemcpyDeviceToDevice, s)) != cudaSuccess) return e;
        if ((e = sgemm('T', 'N', r, m, n, 1.f, Ub, n, X, n, 0.f, w.UtX, r, s)) != cudaSuccess) return e;
        if ((e = sgemm('N', 'N', n, m, r, -1.f, Ub, n, w.UtX, r, 1.f, w.R, n, s)) != cudaSuccess) return e;
        count_launch();
        sumsq_kernel<<<64, 256, 0, s>>>(w.R, nm, sc);
        count_launch();
        sumsq_kernel<<<64, 256, 0, s>>>(X, nm, sc + 1);
        // S = X^T X / s, E = S - I; XE = X E
        if ((e = sgemm('T', 'N', m, m, n, 1.f, X, n, X, n, 0.f, w.G, m, s)) != cudaSuccess) return e;
        count_launch();
        gram_to_e_kernel<<<1, 256, 0, s>>>(w.G, m, sc, w.E, sc + 2);
        if ((e = sgemm('N', 'N', n, m, m, 1.f, X, n, w.E, m, 0.f, w.XE, n, s)) != cudaSuccess) return e;
        count_launch();
        loss_combine_kernel<<<128, 256, 0, s>>>(w.R, X, w.XE, nm, m, mu, B, sc, sc + 2, gX, loss_dev);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    // backward through the layers; gZ (B x m x n) is dL/dZ in the activation layout
    const float *g = w.gZ;
    for (int l = net.depth - 1; l >= 0; --l) {
        const int ci = net.chan[l], co = net.chan[l + 1];
        const float *W = params + net.w_offset(l);
        float *gW = grad + net.w_offset(l);
        float *gb = gW + (size_t)co * ci * net.K;
        const float *in = (l == 0) ? x : w.acts + (size_t)(l - 1) * B * net.width * n;
        count_launch();
        conv_bwd_weight_kernel<<<co * ci, 256, 0, s>>>(g, co, in, ci, n, net.K, B, gW, gb);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if (l > 0) {
            float *gin = (g == w.g0) ? w.g1 : w.g0;
            dim3 grid(blocks_for(n, 128), (ci + kOutPerThread - 1) / kOutPerThread, B);
            count_launch();
            conv_bwd_data_kernel<<<grid, 128, 0, s>>>(g, co, W, in, gin, ci, n, net.K);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            g = gin;
        }
    }
    return cudaSuccess;
}

cudaError_t sketchnet_adam(const SketchNet &net, float *params, const float *grad, float *m1, float *m2, int t,
                           float lr, cudaStream_t s)
{
    const int64_t np = net.num_params();
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = (float)(1.0 - pow(0.9, t)), c2 = (float)(1.0 - pow(0.999, t));
    count_launch();
    adam_kernel<<<blocks_for(np, 256), 256, 0, s>>>(params, grad, m1, m2, np, lr, b1, b2, 1e-8f, c1, c2);
    return cudaGetLastError();
}

cudaError_t sketchnet_input(const double *traj, int T, int64_t n, int C, float *x, double *st, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(st, 0, 2 * sizeof(double), s);
    if (e != cudaSuccess) return e;
    const unsigned grid = blocks_for((size_t)n * C, 256) < 1024 ? blocks_for((size_t)n * C, 256) : 1024;
    count_launch();
    snapshot_kernel<<<grid, 256, 0, s>>>(traj, T, n, C, x, st);
    count_launch();
    standardise_kernel<<<grid, 256, 0, s>>>(traj, T, n, C, x, st);
    return cudaGetLastError();
}

cudaError_t sumsq(const float *x, size_t n, double *out, cudaStream_t s)
{
    count_launch();
    sumsq_kernel<<<64, 256, 0, s>>>(x, n, out);
    return cudaGetLastError();
}

}  // namespace riot
