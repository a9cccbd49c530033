"""Plain FP64 CPU oracle for the FM-CFUST EM algorithm (arXiv:1606.02054).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  The CUDA
library never links, loads or calls it, and it shares no code with the CUDA
path: the only common ground is the seeded synthetic inputs and published
definitions (SplitMix64, Korobov lattices) that each side implements itself.

The C source ``cfust_oracle.c`` follows the paper equation by equation:
eqs (3)-(4) density, (12)-(17) E-step, (18)-(22) M-step, (24)-(26) Aitken,
(27) log-likelihood.  This module only compiles it and marshals numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cfust_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

DEFAULT_NTHREADS = max(1, os.cpu_count() or 1)


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liboracle.so`` (gcc, OpenMP)."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "cfust_oracle.h"))
    ):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-std=gnu11", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Qmc(C.Structure):
    _fields_ = [("npoints", C.c_int), ("nshifts", C.c_int), ("korobov_a", C.c_int),
                ("seed", C.c_uint64), ("moments", C.c_int), ("elogw", C.c_int)]


_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = C.CDLL(path)
            d, i = C.c_double, C.c_int
            L.ora_digamma.argtypes = [d]; L.ora_digamma.restype = d
            L.ora_phi.argtypes = [d]; L.ora_phi.restype = d
            L.ora_phi_inv.argtypes = [d]; L.ora_phi_inv.restype = d
            L.ora_incbeta.argtypes = [d, d, d]; L.ora_incbeta.restype = d
            L.ora_incgamma_p.argtypes = [d, d]; L.ora_incgamma_p.restype = d
            L.ora_chi2_quantile.argtypes = [d, d, d]; L.ora_chi2_quantile.restype = d
            L.ora_t1pdf.argtypes = [d, d]; L.ora_t1pdf.restype = d
            L.ora_t1cdf.argtypes = [d, d]; L.ora_t1cdf.restype = d
            L.ora_t2cdf.argtypes = [d, d, d, d]; L.ora_t2cdf.restype = d
            L.ora_phi2.argtypes = [d, d, d]; L.ora_phi2.restype = d
            L.ora_splitmix64_u01.argtypes = [C.c_uint64]; L.ora_splitmix64_u01.restype = d
            L.ora_qmc_shift.argtypes = [C.POINTER(Qmc), i, i]; L.ora_qmc_shift.restype = d
            L.ora_tkcdf.argtypes = [i, _dp, _dp, d, C.POINTER(Qmc), _dp]
            L.ora_tkcdf.restype = d
            L.ora_tk_moments.argtypes = [i, _dp, _dp, d, C.POINTER(Qmc), _dp, _dp]
            L.ora_tk_joint.argtypes = [i, _dp, _dp, d, d, C.POINTER(Qmc), _dp, _dp]
            L.ora_tk_joint.restype = d
            L.ora_tk_moments.restype = d
            L.ora_pair.argtypes = [i, i, _dp, _dp, _dp, _dp, d, C.POINTER(Qmc), _dp, _dp, _dp,
                                   _dp, _dp, _dp]
            L.ora_pair.restype = i
            L.ora_estep.argtypes = [i, i, i, i, _dp, _dp, _dp, _dp, _dp, _dp, C.POINTER(Qmc),
                                    i, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp]
            L.ora_estep.restype = i
            L.ora_loglik.argtypes = [i, i, i, i, _dp, _dp, _dp, _dp, _dp, _dp, C.POINTER(Qmc),
                                     i, _dp]
            L.ora_loglik.restype = i
            L.ora_mstep.argtypes = [i, i, i, i, _dp, _dp, _dp, _dp, _dp, _dp, d, d, _dp, _dp,
                                    _dp, _dp, _dp, _ip]
            L.ora_mstep.restype = i
            L.ora_mstep_hold.argtypes = [i, i, i, i, _dp, _dp, _dp, _dp, _dp, _dp, d, d, _dp, _dp,
                                         _dp, _dp, _dp, _ip, i]
            L.ora_mstep_hold.restype = i
            L.ora_nu_root.argtypes = [d, d, d, d, _ip]; L.ora_nu_root.restype = d
            L.ora_fit.argtypes = [i, i, i, i, _dp, _dp, _dp, _dp, _dp, _dp, C.POINTER(Qmc), i, d,
                                  d, d, i, _ip, _dp]
            L.ora_fit.restype = i
            L.ora_fit_hold.argtypes = [i, i, i, i, _dp, _dp, _dp, _dp, _dp, _dp, C.POINTER(Qmc), i,
                                       d, d, d, i, _ip, _dp, i]
            L.ora_fit_hold.restype = i
            L.ora_random_partition.argtypes = [i, i, C.c_uint64, i, _ip]
            L.ora_random_partition.restype = None
            L.ora_kmeans.argtypes = [i, i, i, _dp, i, C.c_uint64, i, _ip, _ip, _dp]
            L.ora_kmeans.restype = i
            L.ora_moment_start.argtypes = [i, i, i, i, _dp, _ip, d, d, _dp, _dp, _dp, _dp, _dp]
            L.ora_moment_start.restype = i
            L.ora_init.argtypes = [i, i, i, i, _dp, i, _ip, C.c_uint64, i, _dp, d, C.POINTER(Qmc),
                                   i, _dp, _ip, _dp, _dp, _dp, _dp, _dp]
            L.ora_init.restype = i
            L.ora_aitken_converged.argtypes = [d, d, d, d, _dp]
            L.ora_aitken_converged.restype = i
            _lib = L
    return _lib


def _ptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(_dp)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def qmc(npoints=1024, nshifts=8, korobov_a=119, seed=0, moments=0, elogw=0):
    """Lattice settings (both sides receive the same values as inputs);
    moments = 1 selects the single-pass ratio estimators of the truncated-t
    moments (q >= 3); elogw = 1 (with moments = 1) the exact E[log W | y] from
    the same pass instead of the one-step-late eq (15)."""
    return Qmc(int(npoints), int(nshifts), int(korobov_a), int(seed), int(moments), int(elogw))


# ---- scalar special functions -------------------------------------------------
def digamma(x): return lib().ora_digamma(float(x))
def phi(x): return lib().ora_phi(float(x))
def phi_inv(p): return lib().ora_phi_inv(float(p))
def incbeta(a, b, x): return lib().ora_incbeta(float(a), float(b), float(x))
def incgamma_p(a, x): return lib().ora_incgamma_p(float(a), float(x))
def chi2_quantile(w, nu, wc=None):
    return lib().ora_chi2_quantile(float(w), float(1.0 - w if wc is None else wc), float(nu))
def t1pdf(x, nu): return lib().ora_t1pdf(float(x), float(nu))
def t1cdf(x, nu): return lib().ora_t1cdf(float(x), float(nu))
def t2cdf(h, k, rho, nu): return lib().ora_t2cdf(float(h), float(k), float(rho), float(nu))
def phi2(h, k, rho): return lib().ora_phi2(float(h), float(k), float(rho))
def splitmix64_u01(key): return lib().ora_splitmix64_u01(int(key) & 0xFFFFFFFFFFFFFFFF)
def qmc_shift(spec: Qmc, m, d): return lib().ora_qmc_shift(C.byref(spec), int(m), int(d))


def tkcdf(b, V, nu, spec: Qmc | None = None):
    """T_k(b; 0, V, nu) -> (value, standard error)."""
    b = _f64(b).ravel()
    k = b.size
    V = _f64(V).reshape(k, k)
    spec = spec or qmc()
    se = C.c_double(0.0)
    v = lib().ora_tkcdf(k, _ptr(b), _ptr(V), float(nu), C.byref(spec), C.byref(se))
    return v, se.value


def tk_moments(b, V, nu, spec: Qmc | None = None):
    """(alpha, E[X | X <= b], E[X X^T | X <= b]) for X ~ t_k(0, V, nu), ratio estimators."""
    b = _f64(b).ravel()
    k = b.size
    V = _f64(V).reshape(k, k)
    spec = spec or qmc()
    m1, m2 = np.zeros(k), np.zeros((k, k))
    a = lib().ora_tk_moments(k, _ptr(b), _ptr(V), float(nu), C.byref(spec), _ptr(m1), _ptr(m2))
    return a, m1, m2


def tk_joint(c, Lam, nud, k1, spec: Qmc | None = None):
    """The single-pass estimator sharing alpha_s's lattice pass: (alpha at dof k1 + 2,
    E[X | X <= c], E[X X^T | X <= c]) for X ~ t_k(0, (nud/(k1+2)) Lam, k1 + 2)."""
    c = _f64(c).ravel()
    k = c.size
    Lam = _f64(Lam).reshape(k, k)
    spec = spec or qmc()
    m1, m2 = np.zeros(k), np.zeros((k, k))
    a = lib().ora_tk_joint(k, _ptr(c), _ptr(Lam), float(nud), float(k1), C.byref(spec), _ptr(m1), _ptr(m2))
    return a, m1, m2


def pair(y, mu, Sigma, Delta, nu, spec: Qmc | None = None):
    """One (observation, component) pair: dict(logf, u, elogu, eu, euu, se)."""
    y, mu, Sigma, Delta = _f64(y).ravel(), _f64(mu).ravel(), _f64(Sigma), _f64(Delta)
    p = y.size
    q = Delta.size // p
    spec = spec or qmc()
    logf, u, el, se = (C.c_double() for _ in range(4))
    eu = np.zeros(q)
    euu = np.zeros((q, q))
    rc = lib().ora_pair(p, q, _ptr(y), _ptr(mu), _ptr(Sigma), _ptr(Delta), float(nu),
                        C.byref(spec), C.byref(logf), C.byref(u), C.byref(el), _ptr(eu),
                        _ptr(euu), C.byref(se))
    if rc:
        raise RuntimeError(f"ora_pair failed ({rc})")
    return dict(logf=logf.value, u=u.value, elogu=el.value, eu=eu, euu=euu, se=se.value)


def _params(params):
    pi = _f64(params["pi"])
    mu = _f64(params["mu"])
    Sigma = _f64(params["Sigma"])
    Delta = _f64(params["Delta"])
    nu = _f64(params["nu"])
    return pi, mu, Sigma, Delta, nu


def estep(y, params, spec: Qmc | None = None, nthreads=None):
    """Full E-step: dict(logf, tau, u, elogu, eu, euu, se, loglik), arrays [h, j, ...]."""
    y = _f64(y)
    n, p = y.shape
    pi, mu, Sigma, Delta, nu = _params(params)
    g = pi.size
    q = Delta.shape[-1]
    spec = spec or qmc()
    out = dict(logf=np.zeros((g, n)), tau=np.zeros((g, n)), u=np.zeros((g, n)),
               elogu=np.zeros((g, n)), eu=np.zeros((g, n, q)), euu=np.zeros((g, n, q, q)),
               se=np.zeros((g, n)))
    L = C.c_double()
    rc = lib().ora_estep(n, p, q, g, _ptr(y), _ptr(pi), _ptr(mu), _ptr(Sigma), _ptr(Delta),
                         _ptr(nu), C.byref(spec), int(nthreads or DEFAULT_NTHREADS),
                         _ptr(out["logf"]), _ptr(out["tau"]), _ptr(out["u"]),
                         _ptr(out["elogu"]), _ptr(out["eu"]), _ptr(out["euu"]),
                         _ptr(out["se"]), C.byref(L))
    if rc:
        raise RuntimeError(f"ora_estep failed ({rc})")
    out["loglik"] = L.value
    return out


def loglik(y, params, spec: Qmc | None = None, nthreads=None):
    y = _f64(y)
    n, p = y.shape
    pi, mu, Sigma, Delta, nu = _params(params)
    g, q = pi.size, Delta.shape[-1]
    spec = spec or qmc()
    L = C.c_double()
    rc = lib().ora_loglik(n, p, q, g, _ptr(y), _ptr(pi), _ptr(mu), _ptr(Sigma), _ptr(Delta),
                          _ptr(nu), C.byref(spec), int(nthreads or DEFAULT_NTHREADS), C.byref(L))
    if rc:
        raise RuntimeError(f"ora_loglik failed ({rc})")
    return L.value


HOLD_DELTA, HOLD_NU = 1, 2


def mstep(y, e, params, nu_min=1.0, nu_max=200.0, hold=0):
    """M-step from E-step arrays; returns (new params dict, nu_flag).  hold: HOLD_DELTA
    and/or HOLD_NU keep those parameters at their current values."""
    y = _f64(y)
    n, p = y.shape
    pi, mu, Sigma, Delta, nu = (a.copy() for a in _params(params))
    g, q = pi.size, Delta.shape[-1]
    flag = np.zeros(g, dtype=np.int32)
    rc = lib().ora_mstep_hold(n, p, q, g, _ptr(y), _ptr(_f64(e["tau"])), _ptr(_f64(e["u"])),
                              _ptr(_f64(e["elogu"])), _ptr(_f64(e["eu"])), _ptr(_f64(e["euu"])),
                              float(nu_min), float(nu_max), _ptr(pi), _ptr(mu), _ptr(Sigma),
                              _ptr(Delta), _ptr(nu), flag.ctypes.data_as(_ip), int(hold))
    if rc:
        raise RuntimeError(f"ora_mstep failed ({rc})")
    return dict(pi=pi, mu=mu, Sigma=Sigma, Delta=Delta, nu=nu), flag


def nu_root(n_h, s_h, nu_min=1.0, nu_max=200.0):
    fl = C.c_int(0)
    v = lib().ora_nu_root(float(n_h), float(s_h), float(nu_min), float(nu_max), C.byref(fl))
    return v, fl.value


def aitken_converged(l_km1, l_k, l_kp1, eps):
    li = C.c_double()
    c = lib().ora_aitken_converged(float(l_km1), float(l_k), float(l_kp1), float(eps),
                                   C.byref(li))
    return bool(c), li.value


def fit(y, params, iters, spec: Qmc | None = None, tol=0.0, nu_min=1.0, nu_max=200.0,
        nthreads=None, hold=0):
    """EM fit; returns (params, loglik history [iters_done+1], iters_done)."""
    y = _f64(y)
    n, p = y.shape
    pi, mu, Sigma, Delta, nu = (a.copy() for a in _params(params))
    g, q = pi.size, Delta.shape[-1]
    spec = spec or qmc()
    hist = np.full(iters + 1, np.nan)
    done = C.c_int(0)
    rc = lib().ora_fit_hold(n, p, q, g, _ptr(y), _ptr(pi), _ptr(mu), _ptr(Sigma), _ptr(Delta),
                            _ptr(nu), C.byref(spec), int(iters), float(tol), float(nu_min),
                            float(nu_max), int(nthreads or DEFAULT_NTHREADS), C.byref(done),
                            _ptr(hist), int(hold))
    if rc:
        raise RuntimeError(f"ora_fit failed ({rc})")
    k = done.value
    return dict(pi=pi, mu=mu, Sigma=Sigma, Delta=Delta, nu=nu), hist[: k + 1], k


# ---- initialisation (Sec. 3.3, Algorithm 1, eq 23) ---------------------------
ALPHAS = tuple(round(0.1 * k, 1) for k in range(1, 10))


def random_partition(n, g, seed, start):
    lab = np.zeros(int(n), dtype=np.int32)
    lib().ora_random_partition(int(n), int(g), int(seed) & 0xFFFFFFFFFFFFFFFF, int(start),
                               lab.ctypes.data_as(_ip))
    return lab


def kmeans(y, g, nstarts=1, seed=0, max_iter=100):
    """k-means partitions (Lloyd, seeded starting centres; see ora_kmeans): returns
    (labels (nstarts, n), iterations (nstarts,), centres (nstarts, g, p))."""
    y = _f64(y)
    n, p = y.shape
    lab = np.zeros((nstarts, n), dtype=np.int32)
    its = np.zeros(nstarts, dtype=np.int32)
    cen = np.zeros((nstarts, g, p))
    rc = lib().ora_kmeans(n, p, int(g), _ptr(y), int(nstarts), int(seed) & 0xFFFFFFFFFFFFFFFF, int(max_iter),
                          lab.ctypes.data_as(_ip), its.ctypes.data_as(_ip), _ptr(cen))
    if rc:
        raise ValueError("kmeans: fewer observations than clusters")
    return lab, its, cen


def moment_start(y, labels, g, q, alpha, nu0=10.0):
    """Eq (23) per cluster; returns (params, rc) with rc = 0 or 1 + first failing cluster."""
    y = _f64(y)
    n, p = y.shape
    lab = np.ascontiguousarray(labels, dtype=np.int32)
    out = dict(pi=np.zeros(g), mu=np.zeros((g, p)), Sigma=np.zeros((g, p, p)),
               Delta=np.zeros((g, p, q)), nu=np.zeros(g))
    rc = lib().ora_moment_start(n, p, q, g, _ptr(y), lab.ctypes.data_as(_ip), float(alpha),
                                float(nu0), *[_ptr(out[k]) for k in ("pi", "mu", "Sigma", "Delta", "nu")])
    return out, rc


def init(y, g, q, spec: Qmc | None = None, nstarts=4, labels=None, seed=0, alphas=ALPHAS,
         nu0=10.0, nthreads=None):
    """Algorithm 1: returns (best params, loglik per candidate [nstarts, nalpha], best index)."""
    y = _f64(y)
    n, p = y.shape
    spec = spec or qmc()
    al = _f64(alphas)
    lab = None if labels is None else np.ascontiguousarray(labels, dtype=np.int32).reshape(nstarts, n)
    ll = np.zeros((nstarts, al.size))
    best = C.c_int(-1)
    out = dict(pi=np.zeros(g), mu=np.zeros((g, p)), Sigma=np.zeros((g, p, p)),
               Delta=np.zeros((g, p, q)), nu=np.zeros(g))
    rc = lib().ora_init(n, p, q, g, _ptr(y), int(nstarts),
                        None if lab is None else lab.ctypes.data_as(_ip),
                        int(seed) & 0xFFFFFFFFFFFFFFFF, al.size, _ptr(al), float(nu0),
                        C.byref(spec), int(nthreads or DEFAULT_NTHREADS), _ptr(ll), C.byref(best),
                        *[_ptr(out[k]) for k in ("pi", "mu", "Sigma", "Delta", "nu")])
    if rc:
        raise RuntimeError(f"ora_init failed ({rc})")
    return out, ll, best.value
