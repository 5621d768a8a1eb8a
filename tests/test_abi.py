"""The C ABI library loads and exports every function declared in include/pdmrg.h; argument
errors are reported without touching a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pdmrg.h")


def _declared():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(dmrg_[a-z_0-9]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    import paper_1301_3494_gb300 as pd
    if not os.path.exists(pd.LIB_PATH):
        from paper_1301_3494_gb300 import build
        build.build()
    return pd.lib()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 16
    for n in names:
        assert hasattr(lib, n), n


def test_argument_errors_without_gpu(lib):
    import paper_1301_3494_gb300 as pd
    h = ctypes.c_void_p()
    assert lib.dmrg_init_mpo(ctypes.byref(h), None, None) == 1          # DMRG_ERR_ARG
    assert "null" in lib.dmrg_last_error(None).decode()
    assert lib.dmrg_status_string(7).decode() == "bounded device wait ran out"
    assert lib.dmrg_destroy(None) == 0
    # bad precision is rejected before any device work
    bond = pd.Bond([1, -1], {0: 1}, {0: 1}, __import__("numpy").zeros((1, 2, 2, 1)), [0], [0])
    assert lib.dmrg_heff_apply(ctypes.byref(bond.desc), 9, None, None, None, None, None, None) == 1


def test_mpo_flux_rule_is_checked(lib):
    import numpy as np
    import paper_1301_3494_gb300 as pd
    W = np.zeros((1, 2, 2, 1))
    W[0, 0, 1, 0] = 1.0          # |up><down| raises the charge by 2 but both fluxes are 0
    bond = pd.Bond([1, -1], {0: 1}, {0: 1}, W, [0], [0], W, [0])
    st = lib.dmrg_heff_apply(ctypes.byref(bond.desc), 0, 1, 1, 1, 1, None, None)
    assert st == 5                                                       # DMRG_ERR_QN
