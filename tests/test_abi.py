"""The C-ABI library builds, loads and exports every entry point that
include/cfust.h declares (CPU only: no compute call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1606_02054_gb300 import build

    return build.build()


def _declared():
    src = open(os.path.join(ROOT, "include", "cfust.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(cfust_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("cfust_create", "cfust_destroy", "cfust_set_data", "cfust_set_params",
              "cfust_get_params", "cfust_estep", "cfust_mstep", "cfust_loglik", "cfust_fit",
              "cfust_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_default_options(libpath):
    import paper_1606_02054_gb300 as cf

    o = cf.cfust_default_opts()
    assert (o.precision, o.qmc_points, o.qmc_shifts, o.qmc_korobov_a) == (0, 1024, 8, 119)
    assert (o.nu_min, o.nu_max, o.t2_nodes) == (1.0, 200.0, 0)


def test_invalid_sizes_rejected_without_device(libpath):
    import paper_1606_02054_gb300 as cf

    with pytest.raises(cf.CfustError) as e:
        cf.cfust_create(0, 1, 1, 10)
    assert e.value.status == cf.CFUST_EINVAL
    with pytest.raises(cf.CfustError) as e:
        cf.cfust_create(4, 9, 2, 10)
    assert e.value.status == cf.CFUST_EINVAL


def test_no_cpu_fallback(libpath):
    """Without a GPU, creating a context fails with CFUST_ECUDA (no fallback)."""
    import torch

    import paper_1606_02054_gb300 as cf

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(cf.CfustError) as e:
        cf.cfust_create(2, 2, 2, 10)
    assert e.value.status == cf.CFUST_ECUDA
