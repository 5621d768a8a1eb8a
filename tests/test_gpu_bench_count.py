"""The benchmark's algorithmic flop count equals the library's count for the same bond."""
import numpy as np
import pytest

import workloads as wl
from tests import _layout as LY

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
pd = pytest.importorskip("paper_1301_3494_gb300")


def test_bench_flops_match_library():
    import bench
    mpo = wl.heisenberg_square_cylinder(6, 4)
    qn = list(mpo.site.qn)
    bonds = wl.consistent_sectors(wl.bond_sectors(mpo.L, qn, 0, 300, 3.0), qn)
    j = 10
    bl, br = bonds[j], bonds[j + 2]
    rng = np.random.default_rng(0)
    f0, f1, f2 = mpo.flux[j], mpo.flux[j + 1], mpo.flux[j + 2]
    Ld = torch.as_tensor(LY.pack_env(LY.random_env(bl, f0, rng), bl, f0)).cuda()
    Rd = torch.as_tensor(LY.pack_env(LY.random_env(br, f2, rng), br, f2)).cuda()
    n = sum(bl[k[0]] * br[k[0] + qn[k[1]] + qn[k[2]]] for k in LY.psi_keys(bl, br, qn))
    x = torch.randn(n, dtype=torch.float64, device="cuda")
    y = torch.zeros_like(x)
    bond = pd.Bond(qn, bl, br, mpo.W[j], f0, f1, mpo.W[j + 1], f2)
    fl_lib = pd.heff_apply(bond, pd.FP64, Ld.data_ptr(), Rd.data_ptr(), x.data_ptr(), y.data_ptr())
    fl_py = bench.heff_flops(bl, br, qn, mpo.W[j], f0, mpo.W[j + 1], f2)
    assert fl_lib == pytest.approx(fl_py, rel=1e-12)
