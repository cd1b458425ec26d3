// Double-float arithmetic on the FP32 pipe: a value is an unevaluated pair
// h + l of floats (about 48 significant bits).  Sums use Knuth's TwoSum on the
// high parts, products Dekker's product through the FMA residual.  Pairs are
// not renormalised after every operation: the low part only has to stay well
// below the high part, and every error below is relative to the magnitudes
// of the operands (the conditioning of the expression), as in FP64.  The
// intrinsics keep the compiler from contracting a product and a sum into an
// FMA, which would break the error-free transforms.
#pragma once

namespace h2 {
namespace dfl {

struct F2 {
    float h, l;
};

// s + e = a + b exactly (Knuth's TwoSum)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ F2 add(F2 a, F2 b) {
    float s, e;
    two_sum(a.h, b.h, s, e);
    return {s, __fadd_rn(__fadd_rn(a.l, b.l), e)};
}

__device__ __forceinline__ F2 neg(F2 a) { return {-a.h, -a.l}; }

__device__ __forceinline__ F2 sub(F2 a, F2 b) { return add(a, neg(b)); }

// (a.h + a.l)(b.h + b.l) without the product of the low parts
__device__ __forceinline__ F2 mul(F2 a, F2 b) {
    const float p = __fmul_rn(a.h, b.h);
    return {p, __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, __fmaf_rn(a.h, b.h, -p)))};
}

// a times a small integer k (exact residual of the high product)
__device__ __forceinline__ F2 mul_k(F2 a, float k) {
    const float p = __fmul_rn(k, a.h);
    return {p, __fmaf_rn(k, a.l, __fmaf_rn(k, a.h, -p))};
}

// the same value with h the rounded sum (Fast2Sum: |h| >= |l| holds)
__device__ __forceinline__ F2 renorm(F2 a) {
    const float s = __fadd_rn(a.h, a.l);
    return {s, __fsub_rn(a.l, __fsub_rn(s, a.h))};
}

// sum_d a_d b_d
__device__ __forceinline__ F2 dot3(const F2* a, const F2* b) {
    return add(add(mul(a[0], b[0]), mul(a[1], b[1])), mul(a[2], b[2]));
}

// 1/sqrt(r) for r > 0 of normal float range, r renormalised: the hardware
// approximation y0 (relative error below 2^-22) and the Taylor correction of
// (1 - eps)^(-1/2) = 1 + eps/2 + 3 eps^2/8 + O(eps^3), eps = 1 - r y0^2
// formed from the pairs (y0^2 exactly as y2 + y2e); the remaining relative
// error is about (5/16) eps^3 plus the rounding of eps (2^-46 absolute).
__device__ __forceinline__ F2 rsqrt(F2 r) {
    float y0;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y0) : "f"(r.h));
    const float y2 = __fmul_rn(y0, y0);
    const float y2e = __fmaf_rn(y0, y0, -y2);
    const float t = __fmaf_rn(-r.h, y2, 1.0f);
    const float ep = __fsub_rn(t, __fmaf_rn(r.h, y2e, __fmul_rn(r.l, y2)));
    return {y0, __fmul_rn(__fmul_rn(y0, ep), __fmaf_rn(0.375f, ep, 0.5f))};
}

// an FP64 value as a pair (h = fl(x), l = fl(x - h))
__device__ __forceinline__ F2 split(double x) {
    const float h = (float)x;
    return {h, (float)(x - (double)h)};
}

__device__ __forceinline__ double to_double(F2 a) { return (double)a.h + (double)a.l; }

}  // namespace dfl
}  // namespace h2
