// Gaussian sketch on the device (Algorithm 3: Omega ~ N(0, 1)).
//
// Counter-based Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11) with the
// Box-Muller transform.  Stream layout: key = (seed lo, seed hi), counter =
// (call lo, call hi, stream, 0); one call gives four uint32 words w0..w3,
// u_j = (w_j + 0.5) 2^-32, and stream element 4c + r is
//   r=0: sqrt(-2 ln u0) cos(2 pi u1)   r=1: sqrt(-2 ln u0) sin(2 pi u1)
//   r=2: sqrt(-2 ln u2) cos(2 pi u3)   r=3: sqrt(-2 ln u2) sin(2 pi u3).
// Element (i, j) of an n x ncols block is stream element j*n + i.
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace riot {

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k)
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k.x += W0; k.y += W1; }
        const uint32_t hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
        const uint32_t hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

template <typename real>
__global__ void normal_kernel(uint2 key, uint32_t stream, int64_t n, int ncols, int64_t ld, real *out)
{
    const int64_t total = n * (int64_t)ncols;
    const int64_t ncalls = (total + 3) / 4;
    const double two_pi = 6.283185307179586476925286766559;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncalls;
         c += (int64_t)gridDim.x * blockDim.x) {
        const uint4 w = philox4x32_10(make_uint4((uint32_t)c, (uint32_t)((uint64_t)c >> 32), stream, 0u), key);
        const double u0 = ((double)w.x + 0.5) * 2.3283064365386963e-10;
        const double u1 = ((double)w.y + 0.5) * 2.3283064365386963e-10;
        const double u2 = ((double)w.z + 0.5) * 2.3283064365386963e-10;
        const double u3 = ((double)w.w + 0.5) * 2.3283064365386963e-10;
        const double r0 = sqrt(-2.0 * log(u0)), r1 = sqrt(-2.0 * log(u2));
        double s0, c0, s1, c1;
        sincos(two_pi * u1, &s0, &c0);
        sincos(two_pi * u3, &s1, &c1);
        const double z[4] = {r0 * c0, r0 * s0, r1 * c1, r1 * s1};
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int64_t e = 4 * c + r;
            if (e < total) {
                const int64_t j = e / n, i = e - j * n;
                out[j * ld + i] = (real)z[r];
            }
        }
    }
}

cudaError_t normal_launch(uint64_t seed, uint32_t stream, int64_t n, int ncols, int64_t ld, int is_double,
                          void *out, cudaStream_t s)
{
    if (n <= 0 || ncols <= 0) return cudaSuccess;
    const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    const int64_t ncalls = (n * (int64_t)ncols + 3) / 4;
    int blocks = (int)((ncalls + 255) / 256);
    if (blocks > 8192) blocks = 8192;
    if (is_double)
        { count_launch(); normal_kernel<double><<<blocks, 256, 0, s>>>(key, stream, n, ncols, ld, (double *)out); }
    else
        { count_launch(); normal_kernel<float><<<blocks, 256, 0, s>>>(key, stream, n, ncols, ld, (float *)out); }
    return cudaGetLastError();
}

}  // namespace riot
