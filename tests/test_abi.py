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


def test_gauge_and_gemm_entry_points_reject_bad_arguments(lib):
    """Host-side checks of the inverse-canonical, measurement and grouped-GEMM entry points: every
    case below fails before any device memory is touched."""
    import paper_1301_3494_gb300 as pd
    fake = ctypes.c_void_p(256)           # never dereferenced: each call fails its argument checks first
    n = ctypes.c_int(0)
    nl = ctypes.c_longlong(0)
    assert lib.dmrg_inverse_canonical(None) == 1
    assert lib.dmrg_icmps_bond(None, 0, None, None, 0, ctypes.byref(n)) == 1
    assert lib.dmrg_icmps_v(None, 0, None, 0, ctypes.byref(n)) == 1
    assert lib.dmrg_icmps_site(None, 0, None, 0, ctypes.byref(nl)) == 1
    assert lib.dmrg_local_expectations(None, 0, None, None, 0, None, None, None) == 1
    P = (pd.GemmProblem * 1)()
    S = (pd.GemmSegment * 1)()
    P[0] = pd.GemmProblem(4, 4, 0, 1, 0, 4, 1, 4, 1, 1, 4, 0, 0, 1.0)
    S[0] = pd.GemmSegment(0, 0, 4, 0)
    assert lib.dmrg_gemm64(None, 1, None, 0, fake, fake, fake, 0, None, None) == 1     # no problem list
    assert lib.dmrg_gemm64(P, 1, S, 1, fake, fake, fake, 2, None, None) == 1          # unknown mode
    assert lib.dmrg_gemm64(P, 1, S, 1, None, fake, fake, 0, None, None) == 1          # null buffer
    P[0] = pd.GemmProblem(4, 4, 0, 2, 0, 4, 1, 4, 1, 1, 4, 0, 0, 1.0)
    assert lib.dmrg_gemm64(P, 1, S, 1, fake, fake, fake, 0, None, None) == 1          # segments out of range
    P[0] = pd.GemmProblem(4, 4, 0, 1, 0, 4, 1, 4, 1, 1, 4, 0, 0, 1.0)
    S[0] = pd.GemmSegment(0, 0, 0, 0)
    assert lib.dmrg_gemm64(P, 1, S, 1, fake, fake, fake, 0, None, None) == 1          # K = 0
    info = (ctypes.c_int * 3)(7, 7, 7)
    assert lib.dmrg_gemm64(P, 0, S, 0, fake, fake, fake, 0, info, None) == 0          # empty batch: no work
    assert list(info) == [0, 0, 0]


def test_emulation_needs_tensor_cores(lib):
    """Without an sm_103 GPU the emulated mode is refused (DMRG_ERR_STATE) before device access."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present: covered by tests/test_gpu_emu.py")
    import paper_1301_3494_gb300 as pd
    fake = ctypes.c_void_p(256)
    P = (pd.GemmProblem * 1)(pd.GemmProblem(4, 4, 0, 1, 0, 4, 1, 4, 1, 1, 4, 0, 0, 1.0))
    S = (pd.GemmSegment * 1)(pd.GemmSegment(0, 0, 4, 0))
    assert lib.dmrg_gemm64(P, 1, S, 1, fake, fake, fake, 1, None, None) == 8


def test_split_batch_rejects_bad_arguments(lib):
    """dmrg_svd_split_batch: an empty batch does nothing; a negative count, an unknown mode, a
    missing array, a null device buffer or m_max < 1 fail before any device access."""
    import numpy as np
    import paper_1301_3494_gb300 as pd
    bond = pd.Bond([1, -1], {0: 1}, {0: 1}, np.zeros((1, 2, 2, 1)), [0], [0])
    D = (pd.BondDesc * 1)(bond.desc)
    P = ctypes.c_void_p * 1
    fake = P(256)                          # never dereferenced: each call fails its checks first
    mm = (ctypes.c_int * 1)(4)
    nm = (ctypes.c_int * 1)()
    qm = (ctypes.c_int * 8)()
    km = (ctypes.c_int * 8)()
    f = lib.dmrg_svd_split_batch
    assert f(0, None, None, None, 0, None, None, None, 0, None, None, None, None, None) == 0
    assert f(-1, D, fake, mm, 0, fake, fake, fake, 8, nm, qm, km, None, None) == 1
    for mode in (3, 7, -1):
        assert f(1, D, fake, mm, mode, fake, fake, fake, 8, nm, qm, km, None, None) == 1, mode
    assert f(1, D, None, mm, 0, fake, fake, fake, 8, nm, qm, km, None, None) == 1          # no psi array
    assert f(1, D, P(None), mm, 0, fake, fake, fake, 8, nm, qm, km, None, None) == 1       # null psi buffer
    assert f(1, D, fake, (ctypes.c_int * 1)(0), 0, fake, fake, fake, 8, nm, qm, km, None, None) == 1
    assert "m_max" in lib.dmrg_last_error(None).decode()
