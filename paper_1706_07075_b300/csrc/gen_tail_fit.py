"""Fit the polynomial of the device erfc approximation; writes tail_fit.h.

Form (Press et al., Numerical Recipes, Sec. 6.2: erfc by a fitted exponent):
    erfc(x) ~ t * exp(-x^2 + P(t)),   t = 1 / (1 + x/2),   x >= 0,
so P(t) = ln(erfc(x) / t) + x^2 is smooth on t in (0, 1].  The TOF kernel
only needs x = |tau| / (sigma sqrt 2) <= K / sqrt 2 with K <= 8, i.e.
t in [1/(1 + 2 sqrt 2), 1]; P is fitted there in FP64 by least squares on
Chebyshev nodes (the coefficients are this fit's own, from scipy's erfc),
and the degree is the smallest whose FP64 fit error stays below 1e-8.  The
polynomial is in the centred variable s = (t - t_mid) / t_half in [-1, 1],
whose coefficients decay, so its FP32 Horner evaluation stays accurate.

Run:  python paper_1706_07075_b300/csrc/gen_tail_fit.py
"""
import os

import numpy as np
from scipy.special import erfc

HERE = os.path.dirname(os.path.abspath(__file__))
X_MAX = 8.0 / np.sqrt(2.0)
T_MIN = 1.0 / (1.0 + 0.5 * X_MAX)
T_MID = 0.5 * (1.0 + T_MIN)
T_HALF = 0.5 * (1.0 - T_MIN)


def target(t):
    x = 2.0 / t - 2.0
    return np.log(erfc(x) / t) + x * x


def fit(degree, n_nodes=4000):
    k = np.arange(n_nodes)
    nodes = 0.5 * (1 + T_MIN) + 0.5 * (1 - T_MIN) * np.cos(np.pi * (k + 0.5) / n_nodes)
    V = np.vander((nodes - T_MID) / T_HALF, degree + 1, increasing=True)
    coef, *_ = np.linalg.lstsq(V, target(nodes), rcond=None)
    return coef


def max_fit_error(coef):
    t = np.linspace(T_MIN, 1.0, 200001)
    return float(np.max(np.abs(np.polyval(coef[::-1], (t - T_MID) / T_HALF) - target(t))))


def main():
    for degree in range(4, 16):
        coef = fit(degree)
        err = max_fit_error(coef)
        if err < 1e-8:
            break
    lines = ["// Generated by gen_tail_fit.py: P = sum_k c[k] s^k, s = (t - mid) / half, with",
             "// erfc(x) ~ t exp(-x^2 + P), t = 1/(1 + x/2), fitted for 0 <= x <= 8/sqrt(2)",
             f"// (degree {degree}, FP64 fit error {err:.2e} in the exponent).",
             "#pragma once",
             f"#define RECON_TAIL_FIT_DEGREE {degree}",
             f"static constexpr float kTailFitInvHalf = {1.0 / T_HALF:.9e}f;",
             f"static constexpr float kTailFitMidOverHalf = {T_MID / T_HALF:.9e}f;",
             "",
             "// P(s) by Horner's rule with the coefficients as immediates.",
             "__device__ __forceinline__ float tail_fit_poly(float s)",
             "{",
             f"    float p = {coef[-1]:.9e}f;"]
    lines += [f"    p = fmaf(p, s, {c:.9e}f);" for c in coef[-2::-1]]
    lines += ["    return p;", "}", ""]
    with open(os.path.join(HERE, "tail_fit.h"), "w") as f:
        f.write("\n".join(lines))
    print(f"degree {degree}, fit error {err:.2e}")


if __name__ == "__main__":
    main()
