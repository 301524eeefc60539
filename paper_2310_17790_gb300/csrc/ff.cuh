// Float-float ("double-single") arithmetic on the FP32 pipe: a value is the
// unevaluated sum hi + lo of two floats with |lo| <= ulp(hi) / 2, which
// carries about 47 significant bits.  GB300 runs float64 at 1/64 of the FP32
// rate with long dependent latencies, so the Gauss-Newton sums and solve use
// pairs of floats instead and stay within a few float64 ulps of an exact
// float64 computation for the sizes involved.
//
// Building blocks (error-free transformations):
//   two_sum(a, b)       s + e == a + b exactly (Knuth, TAOCP vol. 2, §4.2.2)
//   fast_two_sum(a, b)  the same when |a| >= |b| (Dekker, Numer. Math. 18, 1971)
//   two_prod(a, b)      p + e == a * b exactly, e from one fused multiply-add
// and, from them, addition, multiplication and the reciprocal (one Newton
// step from the float reciprocal).  All roundings are explicit (__fadd_rn,
// __fmul_rn, fmaf), so compiler contraction cannot break the transformations.
#pragma once

namespace nsf {

struct ff {
    float hi, lo;
};

__device__ __forceinline__ ff ff_make(float hi, float lo) { return ff{hi, lo}; }

__device__ __forceinline__ ff two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bp = __fsub_rn(s, a);
    const float ap = __fsub_rn(s, bp);
    const float e = __fadd_rn(__fsub_rn(a, ap), __fsub_rn(b, bp));
    return ff{s, e};
}

__device__ __forceinline__ ff fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return ff{s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ ff two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return ff{p, fmaf(a, b, -p)};
}

// Accurate addition: both components through two_sum, then renormalised.
__device__ __forceinline__ ff ff_add(ff x, ff y) {
    ff s = two_sum(x.hi, y.hi);
    const ff t = two_sum(x.lo, y.lo);
    s = fast_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
    return fast_two_sum(s.hi, __fadd_rn(s.lo, t.lo));
}

__device__ __forceinline__ ff ff_neg(ff x) { return ff{-x.hi, -x.lo}; }

__device__ __forceinline__ ff ff_sub(ff x, ff y) { return ff_add(x, ff_neg(y)); }

__device__ __forceinline__ ff ff_mul(ff x, ff y) {
    ff p = two_prod(x.hi, y.hi);
    float e = fmaf(x.hi, y.lo, p.lo);
    e = fmaf(x.lo, y.hi, e);
    return fast_two_sum(p.hi, e);
}

// Exact product of two floats as a float-float.
__device__ __forceinline__ ff ff_prod(float a, float b) { return two_prod(a, b); }

// 1 / x: fast float reciprocal y0 of x.hi, then one Newton step
// y = y0 + y0 e with the residual e = 1 - x y0 formed by two fused
// multiply-adds (about 2^-46 absolute) and the product y0 e kept exactly.
__device__ __forceinline__ ff ff_rcp(ff x) {
    const float y0 = __fdividef(1.f, x.hi);
    float e = fmaf(-x.hi, y0, 1.f);
    e = fmaf(-x.lo, y0, e);
    const ff p = two_prod(y0, e);
    return fast_two_sum(y0, __fadd_rn(p.hi, p.lo));
}

__device__ __forceinline__ ff ff_from_double(double d) {
    const float hi = (float)d;
    return ff{hi, (float)(d - (double)hi)};
}

__device__ __forceinline__ double ff_to_double(ff x) { return (double)x.hi + (double)x.lo; }

__device__ __forceinline__ bool ff_isfinite(ff x) { return isfinite(x.hi) && isfinite(x.lo); }

__device__ __forceinline__ ff ff_shfl_xor(ff x, int m) {
    return ff{__shfl_xor_sync(0xffffffffu, x.hi, m), __shfl_xor_sync(0xffffffffu, x.lo, m)};
}

// Sum over the 32 lanes of a warp by a butterfly; every lane gets the same
// bits (float-float addition is commutative, so partners agree).
__device__ __forceinline__ ff ff_warp_sum(ff x) {
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) x = ff_add(x, ff_shfl_xor(x, m));
    return x;
}

// The same over lanes 0-15 (lanes 16-31 hold zeros or need not be summed);
// lane 0 gets the sum.
__device__ __forceinline__ ff ff_half_warp_sum(ff x) {
#pragma unroll
    for (int m = 8; m >= 1; m >>= 1) x = ff_add(x, ff_shfl_xor(x, m));
    return x;
}

}  // namespace nsf
