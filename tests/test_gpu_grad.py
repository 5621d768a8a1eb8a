"""GPU backward of the projected Hamiltonian and the energy gradient (FP64):
element-wise against the oracle's gradients, through torch.autograd (gradcheck), and the
Hellmann-Feynman derivatives dE/dh, dE/dJ of the transverse-field Ising chain against the
free-fermion closed form."""
import numpy as np
import pytest

import workloads as wl
from oracle import exact as EX
from oracle import grad as G
from tests import _layout as LY
from tests._gpu import engine_for, load_mps

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

pd = pytest.importorskip("paper_1301_3494_gb300")


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _case(kind, m, seed):
    rng = np.random.default_rng(seed)
    if kind == "chain":
        mpo, j = wl.heisenberg_chain(40), 20
    elif kind == "cyl":
        mpo, j = wl.heisenberg_square_cylinder(6, 4), 11
    else:
        mpo, j = wl.tfim_chain(30, 1.0, 0.7), 15
    qn = list(mpo.site.qn)
    bonds = wl.bond_sectors(mpo.L, qn, 0, m, sigma=None if kind == "tfim" else 3.0)
    bl, br = bonds[j], bonds[j + 2]
    f0, f1, f2 = mpo.flux[j], mpo.flux[j + 1], mpo.flux[j + 2]
    Lenv, Renv = LY.random_env(bl, f0, rng), LY.random_env(br, f2, rng)
    keys = LY.psi_keys(bl, br, qn)
    psi = {k: rng.standard_normal((bl[k[0]], br[k[0] + qn[k[1]] + qn[k[2]]])) for k in keys}
    ybar = {k: rng.standard_normal(v.shape) for k, v in psi.items()}
    return qn, bl, br, mpo.W[j], mpo.W[j + 1], f0, f1, f2, Lenv, Renv, psi, ybar


@pytest.mark.parametrize("kind,m", [("chain", 60), ("cyl", 90), ("tfim", 40)])
def test_heff_backward_matches_oracle(kind, m):
    qn, bl, br, W1, W2, f0, f1, f2, Lenv, Renv, psi, ybar = _case(kind, m, 11)
    ref = G.heff_backward(Lenv, W1, f0, W2, f2, Renv, psi, ybar, qn)
    bond = pd.Bond(qn, bl, br, W1, f0, f1, W2, f2)
    Ld, Rd = _dev(LY.pack_env(Lenv, bl, f0)), _dev(LY.pack_env(Renv, br, f2))
    x, yb = _dev(LY.pack_psi(psi, bl, br, qn)), _dev(LY.pack_psi(ybar, bl, br, qn))
    xb, Lb, Rb = torch.zeros_like(x), torch.zeros_like(Ld), torch.zeros_like(Rd)
    W1b, W2b = pd.heff_backward(bond, Ld.data_ptr(), Rd.data_ptr(), x.data_ptr(), yb.data_ptr(), xb.data_ptr(),
                                Lb.data_ptr(), Rb.data_ptr())
    torch.cuda.synchronize()
    got_x = LY.unpack_psi(xb.cpu().numpy(), bl, br, qn)
    got_L = LY.unpack_env(Lb.cpu().numpy(), bl, f0)
    got_R = LY.unpack_env(Rb.cpu().numpy(), br, f2)
    for got, want in ((got_x, ref[0]), (got_L, ref[1]), (got_R, ref[2])):
        scale = max(np.abs(v).max() for v in want.values()) + 1.0
        for k in want:
            assert np.abs(got[k] - want[k]).max() <= 1e-11 * scale, k
    for got, want in ((W1b, ref[3]), (W2b, ref[4])):
        assert np.abs(got - want).max() <= 1e-11 * (np.abs(want).max() + 1.0)


def test_autograd_gradcheck():
    """torch.autograd.gradcheck (central differences of the GPU forward) on a small bond."""
    from paper_1301_3494_gb300 import autograd as AG
    qn, bl, br, W1, W2, f0, f1, f2, Lenv, Renv, psi, ybar = _case("chain", 12, 3)
    L = _dev(LY.pack_env(Lenv, bl, f0)).requires_grad_()
    R = _dev(LY.pack_env(Renv, br, f2)).requires_grad_()
    x = _dev(LY.pack_psi(psi, bl, br, qn)).requires_grad_()
    W1t = torch.as_tensor(W1.copy()).requires_grad_()
    W2t = torch.as_tensor(W2.copy()).requires_grad_()
    fn = lambda L_, R_, x_, W1_, W2_: AG.heff(qn, bl, br, f0, f1, f2, L_, R_, x_, W1_, W2_)
    # MPO zeros are structural (no gradient), so check W1/W2 through directions on their nonzeros
    assert torch.autograd.gradcheck(lambda L_, R_, x_: fn(L_, R_, x_, W1t.detach(), W2t.detach()), (L, R, x),
                                    eps=1e-6, atol=1e-7, rtol=1e-6)
    mask1 = torch.as_tensor(W1 != 0.0, dtype=torch.float64)
    d1 = torch.randn(W1.shape, dtype=torch.float64) * mask1
    y = fn(L, R, x, W1t, W2t)
    ybar = torch.randn_like(y)
    (g1,) = torch.autograd.grad((y * ybar).sum(), (W1t,))
    eps = 1e-5
    with torch.no_grad():
        yp = fn(L, R, x, W1t + eps * d1, W2t)
        ym = fn(L, R, x, W1t - eps * d1, W2t)
    fd = float(((yp - ym) * ybar).sum()) / (2 * eps)
    assert abs(fd - float((g1 * d1).sum())) <= 1e-7 * (abs(fd) + 1.0)


@pytest.mark.parametrize("h", [0.5, 1.0, 1.5])
def test_tfim_hellmann_feynman_gradient(h):
    """dE/dh and dE/dJ of the open TFIM chain (L = 16, J = 1) from the energy gradient of the
    converged DMRG state against the free-fermion closed form."""
    L, J = 16, 1.0
    mpo = wl.tfim_chain(L, J, h)
    eng = engine_for(pd, mpo)
    load_mps(eng, wl.random_mps(L, mpo.site.qn, mpo.qtot, 8, seed=2), list(mpo.site.qn))
    for m in (16, 32, 64, 64):
        eng.sweep(m)
    Wbar, e = eng.energy_gradient()
    assert abs(e - eng.energy()) <= 1e-10 * abs(e)
    dh = 1e-3

    def dW(Jp, hp, Jm, hm, step):
        Wp, Wm = wl.tfim_chain(L, Jp, hp).W, wl.tfim_chain(L, Jm, hm).W
        return [(a - b) / (2 * step) for a, b in zip(Wp, Wm)]

    dE_dh = sum(float(np.sum(g * d)) for g, d in zip(Wbar, dW(J, h + dh, J, h - dh, dh)))
    dE_dJ = sum(float(np.sum(g * d)) for g, d in zip(Wbar, dW(J + dh, h, J - dh, h, dh)))
    st = 1e-5
    ref_h = (EX.tfim_energy(L, J, h + st) - EX.tfim_energy(L, J, h - st)) / (2 * st)
    ref_J = (EX.tfim_energy(L, J + st, h) - EX.tfim_energy(L, J - st, h)) / (2 * st)
    assert abs(e - EX.tfim_energy(L, J, h)) <= 1e-8 * abs(e)
    assert abs(dE_dh - ref_h) <= 1e-6 * abs(ref_h)
    assert abs(dE_dJ - ref_J) <= 1e-6 * abs(ref_J)
    eng.close()
