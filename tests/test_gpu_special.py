"""GPU: the FP32 normal CDF and inverse of the lattice integrators (own
polynomial fits, see csrc/fit_special_f32.py) against scipy's FP64 values, with
the CUDA library's normcdff / normcdfinvf measured beside them.

Bounds (FP32 evaluation of the fits, emulated on the CPU in
csrc/fit_special_f32.py's terms): Phi 4e-6 relative for a >= -5 and 3e-5 relative
down to a = -13 (the bottom of FP32's normal range) -- the FP32 rounding of
z sqrt(log2 e) and of the exponent dominates;
Phi^-1 1e-6 absolute where |y| <= 1 (the approximate log2 near p = 1/2) and
3e-6 relative beyond, on the inputs
the integrators can pass, p in [1e-37, 1 - 2^-24].
"""
import numpy as np
import pytest
import scipy.special as sp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cf():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1606_02054_gb300 import build

    build.build()
    import paper_1606_02054_gb300 as cf

    return cf


def test_phi_f32(cf):
    a = np.linspace(-13.0, 9.0, 1_000_001).astype(np.float32)
    ref = sp.ndtr(a.astype(np.float64))
    got = cf.cfust_special_f32(0, a).astype(np.float64)
    lib = cf.cfust_special_f32(2, a).astype(np.float64)
    rel = np.abs(got - ref) / ref
    body = a >= -5
    print(f"Phi own: max rel {rel[body].max():.2e} (a >= -5), {rel.max():.2e} (a >= -13); "
          f"normcdff: {(np.abs(lib - ref) / ref)[body].max():.2e}, {(np.abs(lib - ref) / ref).max():.2e}")
    assert rel[body].max() <= 4e-6
    assert rel.max() <= 3e-5
    assert got[-1] == 1.0 and np.all(got >= 0) and np.all(got <= 1)
    # below FP32's normal range the value flushes to (near) zero, never grows
    far = cf.cfust_special_f32(0, np.array([-14.0, -20.0, -40.0, -1e30], np.float32))
    assert np.all(far <= 1.2e-38)


def test_phi_inverse_f32(cf):
    p = np.concatenate([np.logspace(-37, np.log10(0.5), 500_000),
                        np.linspace(0.5, 1.0 - 2.0 ** -24, 500_000)]).astype(np.float32)
    p = np.clip(p, np.float32(1e-37), np.float32(1.0 - 2.0 ** -24))
    ref = sp.ndtri(p.astype(np.float64))
    got = cf.cfust_special_f32(1, p).astype(np.float64)
    lib = cf.cfust_special_f32(3, p).astype(np.float64)
    err = np.abs(got - ref)
    small = np.abs(ref) <= 1
    rel = err[~small] / np.abs(ref[~small])
    lerr = np.abs(lib - ref)
    print(f"Phi^-1 own: max abs {err[small].max():.2e} (|y| <= 1), max rel {rel.max():.2e}; "
          f"normcdfinvf: {lerr[small].max():.2e}, {(lerr[~small] / np.abs(ref[~small])).max():.2e}")
    assert err[small].max() <= 1e-6
    assert rel.max() <= 3e-6
    # Phi^-1(1/2) = x Q with x = log2(-log2 1/2) = 0 (exact unless lg2 is off by an ulp)
    assert abs(cf.cfust_special_f32(1, np.array([0.5], np.float32))[0]) <= 1e-7
