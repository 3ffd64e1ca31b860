// Measured arithmetic peaks of the GPU the library runs on: the denominators of the
// ALU-bound kernels' roofline fractions (the Hessian kernel's FP32 arithmetic and the FP64
// k x k chain), the FP64 latencies that set the chain's serial steps, and the latency and
// accuracy of the refined reciprocal those chains use (rcp_fast).  Throughput
// kernels run eight independent FMA chains per thread on four CTAs of 256 threads per SM
// (enough warps to fill every sub-partition); latency kernels run one dependent chain on one
// thread and read the SM cycle counter.
#include <cuda_runtime.h>

#include "fp64_rcp.cuh"
#include "internal.h"

namespace riot {

namespace {

constexpr int kIlp = 8;

template <typename T>
__global__ void __launch_bounds__(256) fma_tput_kernel(T *out, int iters, T b, T c)
{
    T a[kIlp];
#pragma unroll
    for (int j = 0; j < kIlp; ++j) a[j] = (T)(threadIdx.x + j) * (T)1e-3;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < kIlp; ++j) a[j] = fma(a[j], b, c);
    }
    T s = 0;
#pragma unroll
    for (int j = 0; j < kIlp; ++j) s += a[j];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// op 0: a = fma(a, b, c); 1: a = rsqrt(a) + c; 2: a = c / a + 1; 3: a = rcp_fast(a) + 1
__global__ void fp64_chain_kernel(double *out, long long *cycles, int iters, int op, double b, double c)
{
    double a = 2.0 + threadIdx.x * 1e-3;
    const long long t0 = clock64();
    if (op == 0)
        for (int i = 0; i < iters; ++i) a = fma(a, b, c);
    else if (op == 1)
        for (int i = 0; i < iters; ++i) a = rsqrt(a) + c;
    else if (op == 2)
        for (int i = 0; i < iters; ++i) a = c / a + 1.0;
    else
        for (int i = 0; i < iters; ++i) a = rcp_fast(a) + 1.0;
    const long long t1 = clock64();
    out[threadIdx.x] = a;
    if (threadIdx.x == 0) cycles[0] = t1 - t0;
}

// Largest distance, in ulps of the correctly rounded 1 / x, of rcp_fast(x) over `per` inputs
// per thread: x = +-2^u, u uniform in [-1100, 1100] from a counter-based hash (so the inputs
// outside the approximation's range, which take the division, are covered too), plus +-1,
// the powers of two next to the range limits and the largest and smallest normal doubles.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ double ulp_distance(double a, double b)
{
    if (a == b) return 0.0;
    if (!isfinite(a) || !isfinite(b) || b == 0.0) return 1e300;
    int ex = 0;
    frexp(b, &ex);
    return fabs(a - b) / ldexp(1.0, (ex - 53 < -1074) ? -1074 : ex - 53);
}

__global__ void rcp_accuracy_kernel(double *out, int per)
{
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    double worst = 0.0;
    for (int i = 0; i < per; ++i) {
        const unsigned long long r = splitmix64((unsigned long long)tid * 0x100000001B3ull + (unsigned long long)i);
        const double u = (double)(r >> 11) * 0x1.0p-53;
        double x = exp2((2.0 * u - 1.0) * 1100.0);
        if (r & 1ull) x = -x;
        worst = fmax(worst, ulp_distance(rcp_fast(x), 1.0 / x));
    }
    if (tid == 0) {
        const double special[10] = {1.0, -1.0, 0x1.0p-1000, 0x1.0p-1001, 0x1.fffffffffffffp+1000, 0x1.0p+1000,
                                    0x1.fffffffffffffp+1023, 0x1.0p-1022, 3.0, 0x1.0p+1001};
        for (int j = 0; j < 10; ++j) worst = fmax(worst, ulp_distance(rcp_fast(special[j]), 1.0 / special[j]));
    }
    out[tid] = worst;
}

template <typename T>
cudaError_t time_tput(T *buf, int blocks, int iters, cudaStream_t s, double *tflops)
{
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e;
    if ((e = cudaEventCreate(&e0)) != cudaSuccess) return e;
    if ((e = cudaEventCreate(&e1)) != cudaSuccess) {
        cudaEventDestroy(e0);
        return e;
    }
    float best = 0.f;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {   // the first launch is a warm-up
        cudaEventRecord(e0, s);
        count_launch();
        fma_tput_kernel<T><<<blocks, 256, 0, s>>>(buf, iters, (T)0.999, (T)1e-3);
        cudaEventRecord(e1, s);
        if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
        e = cudaGetLastError();
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && (best == 0.f || ms < best)) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e == cudaSuccess) *tflops = 2.0 * blocks * 256.0 * kIlp * iters / (best * 1e-3) * 1e-12;
    return e;
}

}  // namespace

}  // namespace riot

using namespace riot;

extern "C" riot_status riot_measure_peaks(int32_t device, double *out, int32_t nout)
{
    if (!out || nout < 1) return RIOT_EINVAL;
    if (cudaSetDevice(device) != cudaSuccess) return RIOT_ECUDA;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return RIOT_ECUDA;
    const int blocks = 4 * sms;
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return RIOT_ECUDA;
    void *buf = nullptr;
    long long *cyc = nullptr;
    double vals[7] = {0, 0, 0, 0, 0, 0, 0};
    cudaError_t e = cudaMalloc(&buf, sizeof(double) * (size_t)blocks * 256);
    if (e == cudaSuccess) e = cudaMalloc(&cyc, sizeof(long long));
    // about 5 ms per FP64 launch and 2 ms per FP32 launch on a 152-SM GPU
    if (e == cudaSuccess) e = time_tput<double>((double *)buf, blocks, 2048, s, &vals[0]);
    if (e == cudaSuccess) e = time_tput<float>((float *)buf, blocks, 65536, s, &vals[1]);
    const int chain_iters[4] = {4096, 512, 512, 512};
    const int slot[4] = {2, 3, 4, 5};
    for (int op = 0; op < 4 && e == cudaSuccess; ++op) {
        count_launch();
        fp64_chain_kernel<<<1, 1, 0, s>>>((double *)buf, cyc, chain_iters[op], op, 0.999, op == 2 ? 1.5 : 1e-3);
        long long c = 0;
        if ((e = cudaGetLastError()) == cudaSuccess) e = cudaMemcpyAsync(&c, cyc, sizeof(c), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        vals[slot[op]] = (double)c / chain_iters[op];
    }
    if (e == cudaSuccess) {   // rcp_fast against the correctly rounded division, 2^24 inputs
        count_launch();
        rcp_accuracy_kernel<<<blocks, 256, 0, s>>>((double *)buf, (1 << 24) / (blocks * 256) + 1);
        e = cudaGetLastError();
        std::vector<double> h((size_t)blocks * 256);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h.data(), buf, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        double worst = 0.0;
        for (double v : h) worst = (v > worst) ? v : worst;
        vals[6] = worst;
    }
    if (buf) cudaFree(buf);
    if (cyc) cudaFree(cyc);
    cudaStreamDestroy(s);
    if (e != cudaSuccess) return RIOT_ECUDA;
    for (int i = 0; i < nout && i < 7; ++i) out[i] = vals[i];
    return RIOT_OK;
}
