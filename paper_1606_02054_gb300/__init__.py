"""GB300 (sm_103a) FM-CFUST EM hot path: Python binding of include/cfust.h.

The functions below carry the C names and only marshal arguments (numpy
arrays or torch tensors in, numpy arrays out); every step of the E- and
M-steps runs in the CUDA library ``libcfust.so`` built by ``build.py``.
There is no CPU fallback: if the library is missing or no GPU is usable the
calls raise ``CfustError``.

Paper: Lee, Leemaqz & McLachlan, "A simple multithreaded implementation of
the EM algorithm for mixture models" (arXiv:1606.02054), Secs. 2-4.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcfust.so")

# cfust_status
CFUST_OK, CFUST_EINVAL, CFUST_ENOTPD, CFUST_EEMPTY, CFUST_ENUROOT = 0, 1, 2, 3, 4
CFUST_ENAN, CFUST_ETIMEOUT, CFUST_ECUDA, CFUST_ENOMEM, CFUST_ESTATE = 5, 6, 7, 8, 9
STATUS_NAMES = {0: "CFUST_OK", 1: "CFUST_EINVAL", 2: "CFUST_ENOTPD", 3: "CFUST_EEMPTY",
                4: "CFUST_ENUROOT", 5: "CFUST_ENAN", 6: "CFUST_ETIMEOUT", 7: "CFUST_ECUDA",
                8: "CFUST_ENOMEM", 9: "CFUST_ESTATE"}
CFUST_PREC_FP64, CFUST_PREC_FP32, CFUST_PREC_MIXED = 0, 1, 2
CFUST_FIT_NO_FINAL = 1
CFUST_HOLD_DELTA, CFUST_HOLD_NU = 1, 2
CFUST_MODEL_CFUST, CFUST_MODEL_CFUSN = 0, 1
CFUST_F32, CFUST_F64 = 0, 1
CFUST_MLP_IN, CFUST_MLP_H, CFUST_MLP_OUT, CFUST_MLP_NPARAM, CFUST_MLP_NSTAT = 48, 256, 48, 156464, 288
# kernel classes of cfust_profile
PROF_NAMES = ("setup", "chi_table", "plan", "level0_Tq", "level1_Tq-1", "level2_Tq-2",
              "moments_Tq", "combine", "fixup_fp64", "reduce", "mstep", "surrogate")
CFUST_NPROF = len(PROF_NAMES)


class CfustError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class cfust_surrogate_opts(C.Structure):
    _fields_ = [("epochs", C.c_int), ("batch", C.c_int), ("samples_per_epoch", C.c_int64),
                ("lr", C.c_float), ("margin", C.c_float), ("seed", C.c_uint64)]


class cfust_opts(C.Structure):
    _fields_ = [("precision", C.c_int), ("qmc_points", C.c_int), ("qmc_shifts", C.c_int),
                ("qmc_korobov_a", C.c_int), ("seed", C.c_uint64), ("nu_min", C.c_double),
                ("nu_max", C.c_double), ("device", C.c_int), ("cuda_stream", C.c_void_p),
                ("t2_nodes", C.c_int), ("profile", C.c_int), ("moments", C.c_int),
                ("hold", C.c_int), ("model", C.c_int), ("elogw", C.c_int), ("tensor_stats", C.c_int)]


class cfust_rates(C.Structure):
    _fields_ = [("sm_mhz", C.c_double), ("fp32_fma", C.c_double), ("fp64_fma", C.c_double),
                ("mufu_ex2", C.c_double), ("mufu_lg2", C.c_double), ("mufu_rcp", C.c_double),
                ("mix_points", C.c_double * 9), ("t2_nodes", C.c_double)]


class cfust_params(C.Structure):
    _fields_ = [("pi", C.POINTER(C.c_double)), ("mu", C.POINTER(C.c_double)),
                ("Sigma", C.POINTER(C.c_double)), ("Delta", C.POINTER(C.c_double)),
                ("nu", C.POINTER(C.c_double))]


_lock = threading.Lock()
_lib = None
_dp = C.POINTER(C.c_double)


def lib():
    """Load libcfust.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise CfustError(CFUST_ECUDA, f"{LIB_PATH} is missing; build it with "
                                 "`python -m paper_1606_02054_gb300.build`")
            L = C.CDLL(LIB_PATH)
            vp, i, d, i64 = C.c_void_p, C.c_int, C.c_double, C.c_int64
            L.cfust_default_opts.argtypes = [C.POINTER(cfust_opts)]
            L.cfust_default_opts.restype = None
            L.cfust_create.argtypes = [C.POINTER(vp), i, i, i, i64, C.POINTER(cfust_opts)]
            L.cfust_destroy.argtypes = [vp]
            L.cfust_set_data.argtypes = [vp, vp, i, i64, i]
            L.cfust_set_params.argtypes = [vp, C.POINTER(cfust_params)]
            L.cfust_get_params.argtypes = [vp, C.POINTER(cfust_params)]
            L.cfust_estep.argtypes = [vp, _dp]
            L.cfust_get_pairs.argtypes = [vp, _dp, _dp, _dp, _dp, _dp, _dp, _dp]
            L.cfust_get_stats.argtypes = [vp, _dp]
            L.cfust_mstep.argtypes = [vp]
            L.cfust_loglik.argtypes = [vp, _dp]
            L.cfust_fit.argtypes = [vp, i, d, C.POINTER(i), _dp]
            L.cfust_fit_batch.argtypes = [i, C.POINTER(vp), i, d, i, C.POINTER(i), _dp, C.POINTER(i)]
            L.cfust_fit_batch.restype = i
            L.cfust_init.argtypes = [vp, i, vp, C.c_uint64, i, _dp, d, _dp, C.POINTER(i)]
            L.cfust_init.restype = i
            L.cfust_kmeans.argtypes = [vp, i, C.c_uint64, i, vp, C.POINTER(i), _dp]
            L.cfust_kmeans.restype = i
            L.cfust_autotune.argtypes = [vp, i, C.POINTER(i), _dp]
            L.cfust_autotune.restype = i
            L.cfust_special_f32.argtypes = [i, i64, vp, vp, i]
            L.cfust_special_f32.restype = i
            L.cfust_tk_eval.argtypes = [vp, i, i, _dp, _dp, _dp, _dp, _dp]
            L.cfust_last_error.argtypes = [vp]
            L.cfust_last_error.restype = C.c_char_p
            L.cfust_launch_count.argtypes = [vp]
            L.cfust_launch_count.restype = i64
            L.cfust_profile.argtypes = [vp, _dp, C.POINTER(C.c_int64), i]
            L.cfust_profile.restype = i
            L.cfust_profile_work.argtypes = [vp, _dp]
            L.cfust_profile_work.restype = i
            L.cfust_rows_per_segment.argtypes = [i, i, i, i, C.POINTER(i64)]
            L.cfust_rows_per_segment.restype = i
            L.cfust_segment_count.argtypes = [vp, C.POINTER(i64), C.POINTER(i)]
            L.cfust_segment_count.restype = i
            L.cfust_estep_segments.argtypes = [vp, vp, i64]
            L.cfust_estep_segments.restype = i
            L.cfust_reduce_segments.argtypes = [vp, vp, i64, i64, _dp]
            L.cfust_reduce_segments.restype = i
            L.cfust_aitken_converged.argtypes = [d, d, d, d]
            L.cfust_aitken_converged.restype = i
            L.cfust_debug_read.argtypes = [vp, i, vp, i64, C.POINTER(C.c_int64)]
            L.cfust_debug_read.restype = i
            L.cfust_reduce_stats_noalloc.argtypes = [i, i, i, i64] + [vp] * 11
            L.cfust_reduce_stats_noalloc.restype = i
            L.cfust_measure_rates.argtypes = [i, d, C.POINTER(cfust_rates)]
            L.cfust_measure_rates.restype = i
            f32p = C.POINTER(C.c_float)
            L.cfust_mlp_init.argtypes = [C.c_uint64, i, i, vp, i]
            L.cfust_mlp_grad.argtypes = [vp, i64, i, vp, vp, vp, vp, vp, _dp, i]
            L.cfust_mlp_adam.argtypes = [vp, vp, vp, vp, i64, C.c_float, i]
            L.cfust_mlp_records.argtypes = [vp, vp, C.c_float, i, i64, vp, vp, vp, vp, vp, vp, i]
            L.cfust_surrogate_default_opts.argtypes = []
            L.cfust_surrogate_default_opts.restype = cfust_surrogate_opts
            L.cfust_surrogate_train.argtypes = [vp, C.POINTER(cfust_surrogate_opts), _dp, _dp]
            L.cfust_surrogate_use.argtypes = [vp, i]
            L.cfust_surrogate_info.argtypes = [vp, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
            L.cfust_surrogate_params.argtypes = [vp, f32p, f32p]
            for name in ("cfust_mlp_init", "cfust_mlp_grad", "cfust_mlp_adam", "cfust_mlp_records",
                         "cfust_surrogate_train", "cfust_surrogate_use", "cfust_surrogate_info",
                         "cfust_surrogate_params"):
                getattr(L, name).restype = i
            for name in ("cfust_create", "cfust_destroy", "cfust_set_data", "cfust_set_params",
                         "cfust_get_params", "cfust_estep", "cfust_get_pairs", "cfust_get_stats",
                         "cfust_mstep", "cfust_loglik", "cfust_fit", "cfust_tk_eval"):
                getattr(L, name).restype = i
            _lib = L
    return _lib


def _check(status, ctx=None, allow=()):
    if status != CFUST_OK and status not in allow:
        raise CfustError(status, cfust_last_error(ctx))
    return status


def _ptr(a):
    return None if a is None else a.ctypes.data_as(_dp)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class Context:
    """Owns one cfust_ctx (destroyed with the object)."""

    def __init__(self, handle, p, q, g, n):
        self.handle, self.p, self.q, self.g, self.n = handle, p, q, g, n

    @property
    def _as_parameter_(self):
        return self.handle

    def __del__(self):
        h, self.handle = getattr(self, "handle", None), None
        if h and _lib is not None:
            _lib.cfust_destroy(h)


# ---------------------------------------------------------------------------
# the ABI, one function per C entry point
# ---------------------------------------------------------------------------
def cfust_default_opts(**overrides) -> cfust_opts:
    o = cfust_opts()
    lib().cfust_default_opts(C.byref(o))
    for k, v in overrides.items():
        setattr(o, k, v)
    return o


def cfust_create(p, q, g, n, opts: cfust_opts | None = None) -> Context:
    h = C.c_void_p()
    st = lib().cfust_create(C.byref(h), int(p), int(q), int(g), int(n),
                            None if opts is None else C.byref(opts))
    _check(st, None)
    return Context(h.value, int(p), int(q), int(g), int(n))


def cfust_destroy(ctx: Context):
    h, ctx.handle = ctx.handle, None
    return _check(lib().cfust_destroy(h))


def cfust_set_data(ctx: Context, y):
    """y: (n, p) numpy array (host) or torch tensor (host or device), f32 or f64."""
    try:
        import torch
        is_t = isinstance(y, torch.Tensor)
    except ImportError:  # pragma: no cover
        is_t = False
    if is_t:
        if y.dim() != 2 or y.shape[0] != ctx.n or y.shape[1] != ctx.p or y.stride(1) != 1:
            raise CfustError(CFUST_EINVAL, "y must be (n, p) with unit column stride")
        dt = {torch.float32: CFUST_F32, torch.float64: CFUST_F64}.get(y.dtype)
        if dt is None:
            raise CfustError(CFUST_EINVAL, "y must be float32 or float64")
        st = lib().cfust_set_data(ctx.handle, C.c_void_p(y.data_ptr()), dt, int(y.stride(0)),
                                  int(y.is_cuda))
        return _check(st, ctx)
    y = np.asarray(y)
    if y.dtype == np.float32:
        yy, dt = np.ascontiguousarray(y), CFUST_F32
    else:
        yy, dt = _f64(y), CFUST_F64
    if yy.shape != (ctx.n, ctx.p):
        raise CfustError(CFUST_EINVAL, f"y must have shape {(ctx.n, ctx.p)}")
    return _check(lib().cfust_set_data(ctx.handle, yy.ctypes.data_as(C.c_void_p), dt, ctx.p, 0), ctx)


def cfust_set_params(ctx: Context, params):
    arrs = [_f64(params[k]).ravel() for k in ("pi", "mu", "Sigma", "Delta", "nu")]
    P = cfust_params(*[_ptr(a) for a in arrs])
    return _check(lib().cfust_set_params(ctx.handle, C.byref(P)), ctx)


def cfust_get_params(ctx: Context):
    p, q, g = ctx.p, ctx.q, ctx.g
    out = dict(pi=np.zeros(g), mu=np.zeros((g, p)), Sigma=np.zeros((g, p, p)),
               Delta=np.zeros((g, p, q)), nu=np.zeros(g))
    P = cfust_params(*[_ptr(out[k]) for k in ("pi", "mu", "Sigma", "Delta", "nu")])
    _check(lib().cfust_get_params(ctx.handle, C.byref(P)), ctx)
    return out


def cfust_estep(ctx: Context) -> float:
    L = C.c_double()
    _check(lib().cfust_estep(ctx.handle, C.byref(L)), ctx)
    return L.value


def cfust_get_pairs(ctx: Context):
    g, n, q = ctx.g, ctx.n, ctx.q
    out = dict(logf=np.zeros((g, n)), tau=np.zeros((g, n)), u=np.zeros((g, n)),
               elogu=np.zeros((g, n)), eu=np.zeros((g, n, q)), euu=np.zeros((g, n, q, q)),
               se=np.zeros((g, n)))
    _check(lib().cfust_get_pairs(ctx.handle, *[_ptr(out[k]) for k in
                                               ("logf", "tau", "u", "elogu", "eu", "euu", "se")]), ctx)
    return out


def cfust_get_stats(ctx: Context):
    p, q = ctx.p, ctx.q
    S = 3 + p + q + p * q + q * q + p * p
    out = np.zeros(ctx.g * S)
    _check(lib().cfust_get_stats(ctx.handle, _ptr(out)), ctx)
    return out.reshape(ctx.g, S)


def cfust_mstep(ctx: Context) -> int:
    """Returns CFUST_OK or CFUST_ENUROOT (nu clamped); raises on other errors."""
    return _check(lib().cfust_mstep(ctx.handle), ctx, allow=(CFUST_ENUROOT,))


def cfust_loglik(ctx: Context) -> float:
    L = C.c_double()
    _check(lib().cfust_loglik(ctx.handle, C.byref(L)), ctx)
    return L.value


def cfust_fit(ctx: Context, max_iter, tol=0.0):
    """Returns (iterations, log-likelihood history l(Psi^(0..iterations)))."""
    hist = np.full(int(max_iter) + 1, np.nan)
    it = C.c_int(0)
    _check(lib().cfust_fit(ctx.handle, int(max_iter), float(tol), C.byref(it), _ptr(hist)), ctx)
    return it.value, hist[: it.value + 1]


def cfust_fit_batch(ctxs, max_iter, tol=0.0, flags=0):
    """Runs cfust_fit on every context concurrently (one device-controlled graph per fit).

    Returns (iters, hist, status): iters (nfits,), hist (nfits, max_iter+1) with NaN where
    not reached, status (nfits,) of per-fit cfust_status codes (no exception for a failing
    fit; read its message with cfust_last_error)."""
    nf = len(ctxs)
    handles = (C.c_void_p * max(nf, 1))(*[c.handle for c in ctxs])
    iters = np.zeros(nf, dtype=np.int32)
    hist = np.full((nf, int(max_iter) + 1), np.nan)
    status = np.zeros(nf, dtype=np.int32)
    st = lib().cfust_fit_batch(nf, handles, int(max_iter), float(tol), int(flags),
                               iters.ctypes.data_as(C.POINTER(C.c_int)), _ptr(hist),
                               status.ctypes.data_as(C.POINTER(C.c_int)))
    if st != CFUST_OK and not np.any(status != CFUST_OK):
        raise CfustError(st, cfust_last_error(None))
    return iters, hist, status


def cfust_kmeans(ctx: Context, nstarts=1, seed=0, max_iter=100):
    """k-means partitions on the device (see include/cfust.h): (labels (nstarts, n) int32,
    iterations (nstarts,), centres (nstarts, g, p))."""
    lab = np.zeros((int(nstarts), ctx.n), dtype=np.int32)
    its = np.zeros(int(nstarts), dtype=np.int32)
    cen = np.zeros((int(nstarts), ctx.g, ctx.p))
    _check(lib().cfust_kmeans(ctx.handle, int(nstarts), int(seed) & 0xFFFFFFFFFFFFFFFF, int(max_iter),
                              lab.ctypes.data_as(C.c_void_p), its.ctypes.data_as(C.POINTER(C.c_int)),
                              _ptr(cen)), ctx)
    return lab, its, cen


def cfust_autotune(ctx: Context, reps=3):
    """Times the integrators' candidate launch shapes on this context's records and keeps
    the fastest (see include/cfust.h): returns (choices {t2_lanes, mom_points}, timings
    {name: ms or None})."""
    ch = (C.c_int * 2)()
    ms = np.zeros(7)
    _check(lib().cfust_autotune(ctx.handle, int(reps), ch, _ptr(ms)), ctx)
    names = ["t2_lanes_2", "t2_lanes_4", "t2_lanes_8", "t2_lanes_16", "t2_lanes_32", "mom_points_1", "mom_points_2"]
    return ({"t2_lanes": int(ch[0]), "mom_points": int(ch[1])},
            {k: (float(v) if v >= 0 else None) for k, v in zip(names, ms)})


def cfust_init(ctx: Context, nstarts=4, labels=None, seed=0, alphas=None, nu0=10.0):
    """Algorithm 1: sets the context's Psi to the best moment start; returns (loglik per
    candidate [nstarts, nalpha], best index)."""
    al = None if alphas is None else _f64(alphas)
    nal = 9 if al is None else al.size
    lab = None
    if labels is not None:
        lab = np.ascontiguousarray(labels, dtype=np.int32).reshape(nstarts, ctx.n)
    ll = np.zeros((nstarts, nal))
    best = C.c_int(-1)
    _check(lib().cfust_init(ctx.handle, int(nstarts), None if lab is None else lab.ctypes.data,
                            int(seed) & 0xFFFFFFFFFFFFFFFF, 0 if al is None else nal, _ptr(al),
                            float(nu0), _ptr(ll), C.byref(best)), ctx)
    return ll, best.value


def cfust_special_f32(fn, x, device=0):
    """fn 0: Phi, 1: Phi^-1 as the FP32 lattice integrators compute them;
    2 / 3: the CUDA library's normcdff / normcdfinvf."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    y = np.empty_like(x)
    _check(lib().cfust_special_f32(int(fn), x.size, x.ctypes.data, y.ctypes.data, int(device)))
    return y


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def cfust_mlp_init(seed, nin, nout, device=0):
    th = np.empty(CFUST_MLP_NPARAM, dtype=np.float32)
    _check(lib().cfust_mlp_init(int(seed) & 0xFFFFFFFFFFFFFFFF, int(nin), int(nout), th.ctypes.data, int(device)))
    return th


def cfust_mlp_grad(theta, f, t, m, nout, device=0):
    """Returns (grad, y, loss) of the masked loss over rows of standardised features."""
    theta, f, t, m = _f32(theta), _f32(f), _f32(t), _f32(m)
    rows = f.shape[0]
    g = np.empty(CFUST_MLP_NPARAM, dtype=np.float32)
    y = np.empty((rows, CFUST_MLP_OUT), dtype=np.float32)
    loss = C.c_double(0.0)
    _check(lib().cfust_mlp_grad(theta.ctypes.data, rows, int(nout), f.ctypes.data, t.ctypes.data, m.ctypes.data,
                                g.ctypes.data, y.ctypes.data, C.byref(loss), int(device)))
    return g, y, loss.value


def cfust_mlp_adam(theta, grad, m, v, step, lr, device=0):
    """One Adam step; returns new (theta, m, v)."""
    theta, m, v = _f32(theta).copy(), _f32(m).copy(), _f32(v).copy()
    grad = _f32(grad)
    _check(lib().cfust_mlp_adam(theta.ctypes.data, grad.ctypes.data, m.ctypes.data, v.ctypes.data, int(step),
                                float(lr), int(device)))
    return theta, m, v


def cfust_mlp_records(theta, stats, margin, bt, Lc, dof, device=0):
    """The fused inference kernel on records: returns (logT, mom, inbox)."""
    theta, stats = _f32(theta), _f32(stats)
    bt = _f64(bt)
    rows, q = bt.shape
    Lc = _f64(Lc).reshape(rows, q, q)
    dof = _f64(dof).reshape(rows)
    W = q + q * (q + 1) // 2
    logT = np.empty(rows)
    mom = np.empty((rows, W))
    inbox = np.empty(rows, dtype=np.int32)
    _check(lib().cfust_mlp_records(theta.ctypes.data, stats.ctypes.data, float(margin), int(q), rows,
                                   bt.ctypes.data, Lc.ctypes.data, dof.ctypes.data, logT.ctypes.data,
                                   mom.ctypes.data, inbox.ctypes.data, int(device)))
    return logT, mom, inbox


def cfust_surrogate_default_opts(**kw):
    o = lib().cfust_surrogate_default_opts()
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def cfust_surrogate_train(ctx: Context, opts=None, **kw):
    """Returns (loglik of the lattice E-step, per-epoch losses)."""
    o = opts if opts is not None else cfust_surrogate_default_opts(**kw)
    ll = C.c_double(0.0)
    losses = np.zeros(max(o.epochs, 1))
    _check(lib().cfust_surrogate_train(ctx.handle, C.byref(o), C.byref(ll), _ptr(losses)), ctx)
    return ll.value, losses[:o.epochs]


def cfust_surrogate_use(ctx: Context, on):
    _check(lib().cfust_surrogate_use(ctx.handle, int(bool(on))), ctx)


def cfust_surrogate_info(ctx: Context):
    r, f = C.c_int64(0), C.c_int64(0)
    _check(lib().cfust_surrogate_info(ctx.handle, C.byref(r), C.byref(f)), ctx)
    return r.value, f.value


def cfust_surrogate_params(ctx: Context):
    th = np.empty(CFUST_MLP_NPARAM, dtype=np.float32)
    st = np.empty(CFUST_MLP_NSTAT, dtype=np.float32)
    _check(lib().cfust_surrogate_params(ctx.handle, th.ctypes.data_as(C.POINTER(C.c_float)),
                                        st.ctypes.data_as(C.POINTER(C.c_float))), ctx)
    return th, st


def cfust_tk_eval(ctx: Context, b, V, nu):
    """T_k(b; 0, V, nu) per case: b (count, k), V (count, k, k), nu (count)."""
    b = _f64(b)
    count, k = b.shape
    V = _f64(V).reshape(count, k, k)
    nu = _f64(nu).reshape(count)
    out, se = np.zeros(count), np.zeros(count)
    _check(lib().cfust_tk_eval(ctx.handle, k, count, _ptr(b), _ptr(V), _ptr(nu), _ptr(out),
                               _ptr(se)), ctx)
    return out, se


def cfust_last_error(ctx: Context | None = None) -> str:
    h = None if ctx is None else (ctx.handle if isinstance(ctx, Context) else ctx)
    msg = lib().cfust_last_error(h)
    return msg.decode() if msg else ""


def cfust_launch_count(ctx: Context) -> int:
    return int(lib().cfust_launch_count(ctx.handle))


def cfust_profile(ctx: Context, reset=False):
    """{class name: (ms, launches)} accumulated since creation or the last reset."""
    ms = np.zeros(CFUST_NPROF)
    n = np.zeros(CFUST_NPROF, dtype=np.int64)
    _check(lib().cfust_profile(ctx.handle, _ptr(ms), n.ctypes.data_as(C.POINTER(C.c_int64)),
                               int(bool(reset))), ctx)
    return {PROF_NAMES[k]: (float(ms[k]), int(n[k])) for k in range(CFUST_NPROF)}


def cfust_profile_work(ctx: Context):
    """{class name: algorithmic units} since creation or the last profile reset
    (lattice points, T_2 quadrature nodes or T_1 records; see include/cfust.h)."""
    u = np.zeros(CFUST_NPROF)
    _check(lib().cfust_profile_work(ctx.handle, _ptr(u)), ctx)
    return {PROF_NAMES[k]: float(u[k]) for k in range(CFUST_NPROF)}


def cfust_rows_per_segment(p, q, g, precision=CFUST_PREC_FP64) -> int:
    r = C.c_int64(0)
    _check(lib().cfust_rows_per_segment(int(p), int(q), int(g), int(precision), C.byref(r)), None)
    return int(r.value)


def cfust_segment_count(ctx: Context):
    """(segments of this context's rows, doubles per segment)."""
    n, w = C.c_int64(0), C.c_int(0)
    _check(lib().cfust_segment_count(ctx.handle, C.byref(n), C.byref(w)), ctx)
    return int(n.value), int(w.value)


def cfust_estep_segments(ctx: Context, seg):
    """Enqueue the E-step and its segment sums into `seg`, a CUDA float64 tensor of
    shape (nseg_out, width), nseg_out >= the context's segment count."""
    if not (seg.is_cuda and seg.is_contiguous()) or seg.element_size() != 8 or seg.dim() != 2:
        raise CfustError(CFUST_EINVAL, "seg: contiguous 2-D CUDA float64 tensor required")
    _check(lib().cfust_estep_segments(ctx.handle, C.c_void_p(seg.data_ptr()), int(seg.shape[0])), ctx)


def cfust_reduce_segments(ctx: Context, seg, n_total) -> float:
    """Reduce the gathered segments (CUDA float64 tensor (nseg, width), rank order) of
    n_total observations in all; returns l(Psi)."""
    if not (seg.is_cuda and seg.is_contiguous()) or seg.element_size() != 8 or seg.dim() != 2:
        raise CfustError(CFUST_EINVAL, "seg: contiguous 2-D CUDA float64 tensor required")
    L = C.c_double()
    _check(lib().cfust_reduce_segments(ctx.handle, C.c_void_p(seg.data_ptr()), int(seg.shape[0]),
                                       int(n_total), C.byref(L)), ctx)
    return L.value


def cfust_aitken_converged(l_km1, l_k, l_kp1, tol) -> bool:
    return bool(lib().cfust_aitken_converged(float(l_km1), float(l_k), float(l_kp1), float(tol)))


def cfust_debug_read(ctx: Context, what, nbytes=1 << 30, dtype=np.float64):
    """Internal device buffer `what` (see include/cfust.h) as a numpy array."""
    buf = np.zeros(max(1, nbytes // np.dtype(dtype).itemsize), dtype=dtype)
    wr = C.c_int64(0)
    _check(lib().cfust_debug_read(ctx.handle, int(what), buf.ctypes.data_as(C.c_void_p),
                                  buf.nbytes, C.byref(wr)), ctx)
    return buf[: wr.value // np.dtype(dtype).itemsize]


def cfust_reduce_stats_noalloc(p, q, g, n, y, pi, mu, logf, u, elogu, eu, euu, tau, stats,
                               stream=None):
    """Allocation-free reduction: all array arguments are CUDA torch tensors
    (float64, contiguous) on the current device; tau may be None.  Every
    tensor must hold at least the elements the library reads or writes
    (y n*p; pi g; mu g*p; logf, u, elogu, tau g*n; eu g*n*q; euu g*n*q*q;
    stats g*(3+p+q+pq+q^2+p^2)+1): a short one is rejected here, before the
    call, since the library cannot check a device pointer's extent."""
    p, q, g, n = int(p), int(q), int(g), int(n)
    need = {"y": n * p, "pi": g, "mu": g * p, "logf": g * n, "u": g * n, "elogu": g * n,
            "eu": g * n * q, "euu": g * n * q * q, "tau": g * n,
            "stats": g * (3 + p + q + p * q + q * q + p * p) + 1}

    def dp(t, name):
        if t is None:
            return None
        if not (t.is_cuda and t.is_contiguous()) or t.element_size() != 8:
            raise CfustError(CFUST_EINVAL, "device float64 contiguous tensors required")
        if t.numel() < need[name]:
            raise CfustError(CFUST_EINVAL, f"cfust_reduce_stats_noalloc: {name} holds {t.numel()} "
                                           f"elements, {need[name]} needed")
        return C.c_void_p(t.data_ptr())

    if p < 1 or q < 1 or g < 1 or n < 1:
        raise CfustError(CFUST_EINVAL, "cfust_reduce_stats_noalloc: sizes out of range")
    if any(t is None for t in (y, pi, mu, logf, u, elogu, eu, euu, stats)):
        raise CfustError(CFUST_EINVAL, "cfust_reduce_stats_noalloc: NULL device pointer")
    st = lib().cfust_reduce_stats_noalloc(p, q, g, n, dp(y, "y"), dp(pi, "pi"), dp(mu, "mu"),
                                          dp(logf, "logf"), dp(u, "u"), dp(elogu, "elogu"),
                                          dp(eu, "eu"), dp(euu, "euu"), dp(tau, "tau"),
                                          dp(stats, "stats"), None if stream is None else C.c_void_p(stream))
    return _check(st, None)


def cfust_measure_rates(device=0, seconds=1.5):
    """Pipe-rate microbenchmarks of the device (see include/cfust.h): a dict of
    whole-GPU rates per second, mix_points keyed by dimension K = 3..8."""
    r = cfust_rates()
    _check(lib().cfust_measure_rates(int(device), float(seconds), C.byref(r)), None)
    out = {k: float(getattr(r, k)) for k in ("sm_mhz", "fp32_fma", "fp64_fma", "mufu_ex2",
                                             "mufu_lg2", "mufu_rcp", "t2_nodes")}
    out["mix_points"] = {K: float(r.mix_points[K]) for K in range(3, 9)}
    return out


def params_from_workload(params):
    """Copy of a parameter dict as contiguous float64 arrays."""
    return {k: _f64(params[k]).copy() for k in ("pi", "mu", "Sigma", "Delta", "nu")}
