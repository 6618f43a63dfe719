// Generated by gen_tail_fit.py: P = sum_k c[k] s^k, s = (t - mid) / half, with
// erfc(x) ~ t exp(-x^2 + P), t = 1/(1 + x/2), fitted for 0 <= x <= 8/sqrt(2)
// (degree 10, FP64 fit error 9.81e-10 in the exponent).
#pragma once
#define RECON_TAIL_FIT_DEGREE 10
static constexpr float kTailFitInvHalf = 2.707106781e+00f;
static constexpr float kTailFitMidOverHalf = 1.707106781e+00f;

// P(s) by Horner's rule with the coefficients as immediates.
__device__ __forceinline__ float tail_fit_poly(float s)
{
    float p = -8.290926918e-06f;
    p = fmaf(p, s, 9.349489660e-06f);
    p = fmaf(p, s, 6.976630923e-05f);
    p = fmaf(p, s, -1.691698947e-04f);
    p = fmaf(p, s, -3.181114207e-04f);
    p = fmaf(p, s, 1.854378934e-03f);
    p = fmaf(p, s, 6.059056141e-04f);
    p = fmaf(p, s, -2.054105259e-02f);
    p = fmaf(p, s, 4.470319919e-03f);
    p = fmaf(p, s, 5.077644600e-01f);
    p = fmaf(p, s, -4.937375564e-01f);
    return p;
}
