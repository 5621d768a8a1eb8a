"""The allocation-free FP64 matvec entry point (for callers that cannot allocate device memory,
e.g. code whose allocations are owned by an external memory manager) gives the same result as
the regular FP64 matvec entry point, on two calls in a row through the C ABI.

Collected last on purpose, so a run that stops at the first failure has run every other test."""
import numpy as np
import pytest

import workloads as wl
from tests import _layout as LY

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
pd = pytest.importorskip("paper_1301_3494_gb300")


def _case(kind, m, seed):
    rng = np.random.default_rng(seed)
    if kind == "chain":
        mpo, j = wl.heisenberg_chain(40), 20
    else:
        mpo, j = wl.heisenberg_square_cylinder(6, 4), 11
    qn = list(mpo.site.qn)
    bonds = wl.bond_sectors(mpo.L, qn, 0, m, sigma=3.0)
    bl, br = bonds[j], bonds[j + 2]
    f0, f1, f2 = mpo.flux[j], mpo.flux[j + 1], mpo.flux[j + 2]
    bond = pd.Bond(qn, bl, br, mpo.W[j], f0, f1, mpo.W[j + 1], f2)
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a)).cuda()
    Ld = dev(LY.pack_env(LY.random_env(bl, f0, rng), bl, f0))
    Rd = dev(LY.pack_env(LY.random_env(br, f2, rng), br, f2))
    n = sum(bl[k[0]] * br[k[0] + qn[k[1]] + qn[k[2]]] for k in LY.psi_keys(bl, br, qn))
    return bond, Ld, Rd, n


@pytest.mark.parametrize("kind,m", [("chain", 120), ("cyl", 300)])
def test_noalloc_matches_regular_entry_point_twice(kind, m):
    bond, Ld, Rd, n = _case(kind, m, 7)
    gen = torch.Generator(device="cuda").manual_seed(3)
    for _ in range(2):                       # the shared scratch keeps the previous call's data
        x = torch.randn(n, dtype=torch.float64, device="cuda", generator=gen)
        y_ref = torch.zeros_like(x)
        y = torch.full_like(x, float("nan"))  # the entry point must overwrite every element
        pd.heff_apply(bond, pd.FP64, Ld.data_ptr(), Rd.data_ptr(), x.data_ptr(), y_ref.data_ptr())
        pd.heff_apply_noalloc(bond, Ld.data_ptr(), Rd.data_ptr(), x.data_ptr(), y.data_ptr())
        torch.cuda.synchronize()
        scale = y_ref.abs().max().item()
        assert torch.isfinite(y).all()
        assert (y - y_ref).abs().max().item() <= 1e-12 * scale


def test_noalloc_rejects_oversized_bond():
    bond, Ld, Rd, n = _case("cyl", 6000, 8)
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    y = torch.zeros_like(x)
    with pytest.raises(pd.DMRGError) as ei:
        pd.heff_apply_noalloc(bond, Ld.data_ptr(), Rd.data_ptr(), x.data_ptr(), y.data_ptr())
    assert ei.value.status == 4                # DMRG_ERR_CAPACITY
