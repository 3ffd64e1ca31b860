// Reciprocal of a double on the latency-bound FP64 chains (Cholesky pivots, the LU of the
// inverse iteration, Householder reflectors).  On this GPU a dependent FP64 FMA takes 64
// cycles, `1.0 / d` about 430 and a general division about 640; the hardware approximation
// `rcp.approx.ftz.f64` (relative error below 2^-19.9, measured over 4e7 log-uniform inputs)
// takes about 45.  One step of the third-order iteration for 1 / d,
//     e = 1 - d y,   y' = y (1 + e + e^2)    (Householder's method of order 3),
// leaves a truncation error of about e^3 < 2^-59, so the result is within one ulp of the
// correctly rounded reciprocal (measured: at most 1 ulp from `1.0 / d`), in three dependent
// FMAs after the approximation (about 240 cycles).  Inputs whose reciprocal the flush-to-zero
// approximation cannot represent (binary exponent outside [-1000, 1000]), zeros, infinities
// and NaNs take the division instead.
#pragma once

namespace riot {

__device__ __forceinline__ double rcp_fast(double d)
{
    const long long ex = (__double_as_longlong(d) >> 52) & 0x7ff;   // biased binary exponent
    if (ex < 1023 - 1000 || ex > 1023 + 1000) return 1.0 / d;
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(d));
    const double e = fma(-d, y, 1.0);
    return fma(y, fma(e, e, e), y);
}

}  // namespace riot
