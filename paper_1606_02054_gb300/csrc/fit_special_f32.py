"""Derives the coefficients of the FP32 special functions of the integrators
(special.cuh): the normal CDF and its inverse of the lattice integrators
(cf_ncdf_f32, cf_ncdfinv_f32) and the sine of the T_2 quadrature (cf_sin_pi).

Both are this project's own fits (Lawson's iteratively reweighted least
squares in the Chebyshev basis, i.e. a near-minimax polynomial), made in FP64
against scipy.special on a dense grid and printed in the monomial basis of the
mapped variable t in [-1, 1]:

  Phi(a), a <= 0:  z = |a| / sqrt 2,  tau = 1 / (1 + z / 2),
      Phi(a) = tau * 2^(P(t) - z^2 log2 e),   t = affine(tau),
      P(t) ~ log2(erfcx(z) / tau) - 1   (the -1 is the factor 1/2 of
      Phi = erfc / 2), fitted for z in [0, 9.5] (Phi below FP32's normal
      range beyond that);  Phi(a) = 1 - Phi(-a) for a > 0.
  Phi^-1(p), pm = min(p, 1 - p) in [1e-37, 1/2]:
      x = log2(-log2 pm) in [0, 7],  Phi^-1(pm) = x Q(t), t = affine(x)
      (the factor x makes Phi^-1(1/2) = 0 exactly);  Phi^-1(p) = -x Q for p > 1/2.
  sin(x), |x| <= pi:  r = |x| folded to [0, pi/2] (pi - |x| beyond pi/2),
      sin(r) = r S(r^2) with S fitted on [0, (pi/2)^2] (relative error of sin/r),
      then the sign of x.

Run:  python fit_special_f32.py   (prints the constants and the fit errors)
"""
import numpy as np
import scipy.special as sp
from numpy.polynomial import chebyshev as Ch
from numpy.polynomial import polynomial as Pm

LOG2E = 1.0 / np.log(2.0)


def lawson(x, y, deg, lo, hi, iters=80):
    t = (2.0 * x - (lo + hi)) / (hi - lo)
    w = np.ones_like(x)
    for _ in range(iters):
        c = Ch.chebfit(t, y, deg, w=np.sqrt(w))
        e = np.abs(Ch.chebval(t, c) - y)
        w = w * (e + 1e-300)
        w /= w.sum()
    m = Ch.cheb2poly(c)
    return m, np.abs(Pm.polyval(t, m) - y).max()


def fit_ncdf(deg=8, zmax=9.5):
    z = np.linspace(0.0, zmax, 400001)
    tau = 1.0 / (1.0 + 0.5 * z)
    target = np.log2(sp.erfcx(z) / tau) - 1.0
    lo, hi = 1.0 / (1.0 + 0.5 * zmax), 1.0
    m, err = lawson(tau, target, deg, lo, hi)
    # t = tau * A + B
    return m, 2.0 / (hi - lo), -(hi + lo) / (hi - lo), err


def fit_ncdfinv(deg=8, xmax=7.0):
    x = np.linspace(1e-6, xmax, 400001)
    pm = 2.0 ** (-(2.0 ** x))
    target = sp.ndtri(pm)
    m, _ = lawson(x, target / x, deg, 0.0, xmax)
    err = np.abs(x * Pm.polyval(2.0 * x / xmax - 1.0, m) - target).max()
    return m, 2.0 / xmax, -1.0, err


def fit_sin(deg=4):
    r = np.linspace(1e-6, np.pi / 2, 400001)
    t2 = r * r
    hi = (np.pi / 2) ** 2
    m, _ = lawson(t2, np.sin(r) / r, deg, 0.0, hi)
    # monomial coefficients in r^2 itself (t = 2 r^2 / hi - 1 expanded)
    tpoly = Pm.Polynomial([-1.0, 2.0 / hi])
    S = sum(c * tpoly ** k for k, c in enumerate(m))
    coef = S.coef
    err = np.abs(r * Pm.polyval(t2, coef) - np.sin(r)).max()
    return coef, err


if __name__ == "__main__":
    m, A, B, e = fit_ncdf()
    print(f"// Phi: max |error of the log2 exponent| {e:.2e}")
    print(f"t = tau * {A!r}f + {B!r}f")
    print("P =", ", ".join(f"{c:.9e}f" for c in m))
    m, A, B, e = fit_ncdfinv()
    print(f"// Phi^-1: max |error| {e:.2e}  (value = x * Q(t))")
    print(f"t = x * {A!r}f + {B!r}f")
    print("Q =", ", ".join(f"{c:.9e}f" for c in m))
    coef, e = fit_sin()
    print(f"// sin: max |error| {e:.2e}  (value = r * S(r^2), S in powers of r^2)")
    print("S =", ", ".join(f"{c:.9e}f" for c in coef))
