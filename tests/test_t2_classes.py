"""The FP32 T_2 piece classes (internal.cuh t2_lo_class), emulated in FP64 on the host:
on records the bounds were not fitted on, every piece the classes give 8-24 nodes errs by
less than 5e-6 relative to the record's T_2 against 1024-node graded quadrature, and the
classes use fewer nodes than one 24-node set for every piece.  No GPU."""
import importlib.util
import os

import numpy as np
import pytest


HERE = os.path.dirname(os.path.abspath(__file__))
SPEC = importlib.util.spec_from_file_location(
    "fit_t2_classes", os.path.join(HERE, "..", "paper_1606_02054_gb300", "csrc", "fit_t2_classes.py"))
ftc = importlib.util.module_from_spec(SPEC)
SPEC.loader.exec_module(ftc)


@pytest.mark.parametrize("gen,seed", [("main", 41), ("other", 42)])
def test_committed_bounds_on_held_out_records(gen, seed):
    rng = np.random.default_rng(seed)
    sample = ftc.sample_main if gen == "main" else ftc.sample_other
    t = ftc.piece_table(*sample(rng, 3000))
    cls = ftc.classify(t, ftc.COMMITTED)
    err = t[np.arange(len(t)), 3 + cls]
    small = cls < len(ftc.CLASSES)
    nodes = np.array(ftc.CLASSES + (32,))[cls]
    assert small.sum() > 0.9 * len(t)
    assert err[small].max() < 5e-6, err[small].max()
    assert nodes.mean() < 20.0


def test_quadrature_reference_against_oracle_t2():
    """The emulation's reference (1024 graded nodes over the pieces of t2_setup) against the
    oracle's T_2 (adaptive quadrature of another integral form), tails included."""
    import oracle
    rng = np.random.default_rng(7)
    nu, rho, h, k = ftc.sample_main(rng, 200)
    h = np.minimum(h, 12.0)  # the oracle's adaptive rule is slow beyond
    p0, p1, split, zs, C = ftc.pieces(h, k, rho, nu)
    v = C * (ftc.integrate(p0, zs, nu, 1024, graded=True)
             + np.where(split, ftc.integrate(p1, zs, nu, 1024, graded=True), 0.0))
    ref = np.array([oracle.t2cdf(h[i], k[i], rho[i], nu[i]) for i in range(len(nu))])
    keep = ref > 1e-12
    assert keep.sum() > 100
    assert np.max(np.abs(v - ref)[keep] / ref[keep]) < 1e-9
