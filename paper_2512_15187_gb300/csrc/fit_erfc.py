"""Fit the coefficients of the fast complementary error function used by the kernels.

Form (after the Chebyshev-fitted erfc of Numerical Recipes, 2nd ed., Sec. 6.2, with
coefficients fitted here): for a >= 0 and t = 1 / (1 + P_SCALE a),

    erfc(a) / 2 = t * 2^( Q(t) - log2(e) a^2 ),    Q(t) = log2(e) * g(t) - 1,

where g(t) = ln(erfcx(a)) - ln(t) is smooth on t in (0, 1]. Q is a polynomial fitted in
float64 on Chebyshev nodes of t in [T_MIN, 1] by Lawson's iteratively reweighted least
squares, which converges to the minimax (equioscillating) fit; T_MIN corresponds to
a = 9.3, beyond which erfc(a)/2 is below FP32's smallest normal number. Prints the
coefficients (constant term first) and the maximum relative error of the fit.

    python paper_2512_15187_gb300/csrc/fit_erfc.py [degree]
"""
import sys

import numpy as np
from scipy.special import erfcx

P_SCALE = 0.5
A_MAX = 9.3


def fit(deg: int):
    t_min = 1.0 / (1.0 + P_SCALE * A_MAX)
    k = np.arange(4000)
    tt = 0.5 * (1 + t_min) + 0.5 * (1 - t_min) * np.cos(np.pi * (k + 0.5) / k.size)
    a = (1.0 / tt - 1.0) / P_SCALE
    g = np.log(erfcx(a)) - np.log(tt)
    target = g / np.log(2.0) - 1.0
    V = np.vander(tt, deg + 1, increasing=True)
    wts = np.ones_like(tt)
    for _ in range(200):  # Lawson: weights grow where the error is largest
        sw = np.sqrt(wts)
        c, *_ = np.linalg.lstsq(V * sw[:, None], target * sw, rcond=None)
        err = np.abs(V @ c - target)
        wts = wts * err
        wts /= wts.sum()
    a_chk = np.linspace(0, A_MAX, 200001)
    t_chk = 1.0 / (1.0 + P_SCALE * a_chk)
    q = np.polynomial.polynomial.polyval(t_chk, c)
    approx = t_chk * np.exp2(q - a_chk * a_chk / np.log(2.0))
    exact = 0.5 * erfcx(a_chk) * np.exp(-a_chk * a_chk)
    rel = np.max(np.abs(approx - exact) / exact)
    return c, rel


if __name__ == "__main__":
    degs = [int(sys.argv[1])] if len(sys.argv) > 1 else range(5, 11)
    for d in degs:
        c, rel = fit(d)
        print(f"degree {d}: max relative error {rel:.3e}")
        print("  " + ", ".join(f"{v:.9e}f" for v in c))
