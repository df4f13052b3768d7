"""CPU checks of the C-ABI library: it builds, loads and exports every
function declared in include/swcs.h; without a GPU, context creation fails
cleanly with SWCS_ERR_NO_DEVICE (no compute call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def swcs_mod():
    from paper_2411_07920_gb300 import _build
    _build.build()
    from paper_2411_07920_gb300 import swcs
    return swcs


def test_header_declares_the_boundary(swcs_mod):
    names = swcs_mod.declared_symbols()
    for must in ("swcs_create", "swcs_destroy", "swcs_load_hamiltonian", "swcs_apply_ansatz", "swcs_energy",
                 "swcs_pool_gradients", "swcs_energy_grad", "swcs_get_state", "swcs_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(swcs_mod):
    lib = ctypes.CDLL(swcs_mod.LIB_PATH)
    missing = [n for n in swcs_mod.declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing
    # and the binding covers every declared function
    assert set(swcs_mod.declared_symbols()) <= set(swcs_mod._SIGS)


def test_status_codes_match_header(swcs_mod):
    txt = open(os.path.join(ROOT, "include", "swcs.h")).read()
    codes = dict((int(v), k) for k, v in re.findall(r"SWCS_(?:ERR_)?(\w+)\s*=\s*(-?\d+)", txt))
    assert codes == swcs_mod.STATUS


def test_no_device_is_reported_not_crashed(swcs_mod):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    r = swcs_mod.lib.swcs_create(ctypes.byref(h), None)
    assert r == -6 and not h.value
    assert swcs_mod.lib.swcs_last_error(None) == b"no context"
