// Device arithmetic helpers shared by the library's kernels.
#pragma once

namespace h2 {

// 1/sqrt(a) in FP64 for a > 0 of normal range: the hardware approximation
// (PTX rsqrt.approx.ftz.f64) refined by one Newton-Raphson step for
// f(y) = 1/y^2 - a, y <- y + y (1 - a y^2) / 2, which roughly squares the
// relative error of the approximation.  Four FP64 operations after the
// approximation, against about seven for the library rsqrt(double).
__device__ __forceinline__ double rsqrt_nr(double a) {
    double y;
    asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(a));
    const double t = a * y;
    const double e = fma(-t, y, 1.0);
    return fma(0.5 * y, e, y);
}

}  // namespace h2
