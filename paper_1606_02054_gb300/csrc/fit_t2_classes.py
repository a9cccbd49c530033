"""Derives the piece classes of the FP32 T_2 quadrature (internal.cuh: T2_LO_S2_*,
T2_LO_DMAX_*, T2_LO_ZW; t2_lo_class).

T_2(h, k; rho, nu) is integrated over one or two pieces in the angle phi (special.cuh,
t2_setup): the integrand sin^(nu-1)(phi) T_1(zs sin(phi - phi*); nu + 1) has a peak of
width ~ 1/sqrt(nu - 1) and, at the split point phi*, a rise of width ~ 1/|zs|.  A piece of
length L gets Gauss-Legendre with 8, 12, 16, 20 or 24 nodes by its score

    s = L sqrt(nu - 1 + ZW zs^2),

the smallest class whose bound it meets (the two smallest also capped in nu: a piece that
ends at phi = 0 carries phi^(nu-1), integrated exactly only by enough nodes), else 32.

This script, in FP64 with numpy/scipy only:
  1. samples records (nu log-uniform in [4, 64], |rho| < 0.9, h and k uniform in [-8, 8],
     lower tails of h and k down to T_1 = 1e-12, h up to 40) and forms their pieces as the
     kernel does;
  2. integrates every piece with n = 8 .. 32 plain nodes and with 1024 nodes graded toward
     the piece's anchor (the reference), the error relative to the record's T_2;
  3. for each class takes the largest score below which every admissible piece errs by
     less than TOL, and keeps MARGIN of it;
  4. checks the bounds on held-out records of the same and of another distribution.

Run:  python fit_t2_classes.py [records]   (prints the bounds and the held-out errors; the
constants in internal.cuh come from 160,000 training records)
"""
import sys

import numpy as np
from scipy.special import gammaln, stdtr, stdtrit

ZW, TOL, MARGIN = 0.2, 5e-6, 0.85
CLASSES = (8, 12, 16, 20, 24)
DMAX = {8: 20.0, 12: 40.0}  # dof caps of the two smallest classes
# the bounds kept in internal.cuh (T2_LO_S2_c = the square of these)
COMMITTED = {8: 1.54, 12: 4.12, 16: 7.58, 20: 11.32, 24: 15.5}


def gauss_legendre01(n):
    x, w = np.polynomial.legendre.leggauss(n)
    return (x + 1.0) / 2.0, w / 2.0


def pieces(h, k, rho, nu):
    """The angles of t2_setup in FP64: per record the anchor, length and offset of each
    piece, the slope zs and the constant C_nu."""
    sn = np.sqrt(nu)
    sg = np.where(rho > 0, 1.0, -1.0)
    ar = np.abs(rho)
    omr2 = (1.0 - rho) * (1.0 + rho)
    cr = h * ar - sg * k
    phi_h = np.where(h < 0, np.arctan(sn / np.where(h < 0, -h, 1.0)), np.pi / 2 + np.arctan(h / sn))
    phis = np.arctan2(ar * sn, -sg * k)
    D = np.arctan2(sn * cr, sg * h * k + ar * nu)
    split = (rho != 0) & (D > 0)
    zs = -sg * np.sqrt(rho * rho * nu + k * k) * np.sqrt((nu + 1.0) / (omr2 * nu))
    C = np.exp(gammaln((nu + 1.0) / 2.0) - gammaln(nu / 2.0)) / np.sqrt(np.pi)
    anc0 = np.where(split, phis, phi_h)
    p0 = (anc0, -anc0, np.where(split, 0.0, D))
    p1 = (phis, np.where(split, D, 0.0), np.zeros_like(nu))
    return p0, p1, split, zs, C


def integrate(piece, zs, nu, n, graded=False):
    anc, L, d0 = piece
    x, w = gauss_legendre01(n)
    if graded:  # nodes anchor + L u^3, weights 3 u^2
        w = w * 3.0 * x * x
        x = x ** 3
    off = L[:, None] * x[None, :]
    sp = np.sin(anc[:, None] + off)
    sd = np.sin(d0[:, None] + off)
    f = np.exp((nu[:, None] - 1.0) * np.log(np.maximum(sp, 1e-300))) * stdtr(nu[:, None] + 1.0, zs[:, None] * sd)
    return (f * w[None, :]).sum(1) * np.abs(L)


def sample_main(rng, n):
    """The training distribution (and held-out set A)."""
    nu = np.exp(rng.uniform(np.log(4.0), np.log(64.0), n))
    rho = rng.uniform(-0.9, 0.9, n)
    h = rng.uniform(-8.0, 8.0, n)
    k = rng.uniform(-8.0, 8.0, n)
    m = rng.uniform(size=n) < 0.4
    h[m] = stdtrit(nu[m], 10.0 ** rng.uniform(-12.0, -3.0, m.sum()))
    m = rng.uniform(size=n) < 0.25
    k[m] = stdtrit(nu[m], 10.0 ** rng.uniform(-12.0, -3.0, m.sum()))
    m = rng.uniform(size=n) < 0.15
    h[m] = rng.uniform(4.0, 40.0, m.sum())
    return nu, rho, h, k


def sample_other(rng, n):
    """Held-out set B: nu uniform, half the rho near +-0.9, h and k normal, h wide."""
    nu = rng.uniform(4.0, 64.0, n)
    rho = rng.choice([-1.0, 1.0], n) * rng.uniform(0.6, 0.9, n)
    rho[: n // 2] = rng.uniform(-0.9, 0.9, n // 2)
    h = rng.normal(0.0, 2.5, n)
    k = rng.normal(0.0, 2.5, n)
    m = rng.uniform(size=n) < 0.3
    h[m] = rng.uniform(-60.0, 60.0, m.sum())
    return nu, rho, h, k


def piece_table(nu, rho, h, k):
    """One row per piece of a record with T_2 > 1e-12: nu, L, |zs|, then the errors of the
    plain rules with CLASSES + (32,) nodes relative to the record's T_2."""
    p0, p1, split, zs, C = pieces(h, k, rho, nu)
    ref = [integrate(p, zs, nu, 1024, graded=True) for p in (p0, p1)]
    tot = C * (ref[0] + np.where(split, ref[1], 0.0))
    rows = []
    for i, p in enumerate((p0, p1)):
        keep = (tot > 1e-12) & (split if i == 1 else True)
        errs = [C * np.abs(integrate(p, zs, nu, n) - ref[i]) / np.where(tot > 0, tot, 1.0)
                for n in CLASSES + (32,)]
        rows.append(np.column_stack([nu, np.abs(p[1]), np.abs(zs)] + errs)[keep])
    return np.concatenate(rows)


def score(t):
    return t[:, 1] * np.sqrt(t[:, 0] - 1.0 + ZW * t[:, 2] ** 2)


def fit(t):
    s = score(t)
    bounds = {}
    for c, n in enumerate(CLASSES):
        ok = t[:, 0] <= DMAX.get(n, np.inf)
        order = np.argsort(s[ok])
        worst = np.maximum.accumulate(t[ok, 3 + c][order])
        good = np.nonzero(worst < TOL)[0]
        bounds[n] = MARGIN * s[ok][order][good[-1]] if good.size else 0.0
    return bounds


def classify(t, bounds):
    """Class index per piece (len(CLASSES) for the 32-node set), as t2_lo_class."""
    s = score(t)
    cls = np.full(len(t), len(CLASSES))
    for c in reversed(range(len(CLASSES))):
        n = CLASSES[c]
        cls[(s <= bounds[n]) & (t[:, 0] <= DMAX.get(n, np.inf))] = c
    return cls


def main():
    records = int(sys.argv[1]) if len(sys.argv) > 1 else 40000
    train = np.concatenate([piece_table(*sample_main(np.random.default_rng(s), records // 8)) for s in range(1, 9)])
    bounds = fit(train)
    print(f"training pieces: {len(train)}; bounds on s = L sqrt(nu - 1 + {ZW} zs^2) at {TOL:g}, x {MARGIN}:")
    for n in CLASSES:
        cap = f", nu <= {DMAX[n]:g}" if n in DMAX else ""
        print(f"  {n:2d} nodes: s <= {bounds[n]:.2f}{cap}")
    for name, gen, seeds in (("A (same distribution)", sample_main, range(11, 19)),
                             ("B (other distribution)", sample_other, range(21, 29))):
        t = np.concatenate([piece_table(*gen(np.random.default_rng(s), records // 8)) for s in seeds])
        for label, b in (("fitted", bounds), ("internal.cuh", COMMITTED)):
            cls = classify(t, b)
            err = t[np.arange(len(t)), 3 + cls]
            nodes = np.array(CLASSES + (32,))[cls]
            print(f"held-out {name}, {label} bounds: {len(t)} pieces, {nodes.mean():.1f} nodes a piece, "
                  f"worst error of classes 8-24: {err[cls < len(CLASSES)].max():.2e}")


if __name__ == "__main__":
    main()
