"""The C-ABI library builds, loads without a GPU and exports every entry point
that include/lqcd_amg.h declares (no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lqcd_amg.h")


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:amg_status|void|unsigned long long|const char\s*\*)\s*(amg_\w+)\s*\(", text, re.M)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2111_05012_gb300 import capi
    return capi.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["amg_lattice_create", "amg_gauge_create", "amg_dirac_create", "amg_setup", "amg_apply_D",
                     "amg_apply_coarse", "amg_restrict", "amg_prolong", "amg_solve", "amg_last_error"]:
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2111_05012_gb300 import capi
    for name in declared_functions():
        assert hasattr(lib, name), f"{name} not exported by libamg.so"
        assert name in capi.PROTOTYPES, f"{name} has no binding"


def test_binding_has_no_extra_names():
    from paper_2111_05012_gb300 import capi
    assert set(capi.PROTOTYPES) <= set(declared_functions())


def test_params_default_without_gpu(lib):
    from paper_2111_05012_gb300 import capi
    p = capi.amg_params_default()
    assert p.nlevels == 2 and p.sap_iters == 4 and p.mr_iters == 6 and p.outer_m == 16
    assert tuple(p.block[0]) == (4, 4, 4, 4) and p.nvec[0] == 24


def test_invalid_lattice_is_rejected_without_gpu(lib):
    from paper_2111_05012_gb300 import capi
    with pytest.raises(capi.AMGError) as e:
        capi.amg_lattice_create((4, 1, 4, 4))
    assert e.value.status == capi.AMG_EINVAL
    assert "extents" in capi.amg_last_error()
