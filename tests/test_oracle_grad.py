"""The oracle's H_eff gradients against central finite differences of the oracle's matvec.

Phi = <ybar, H_eff(L, W1, W2, R) x> is linear in each argument, so a central difference along a
random direction equals the directional derivative up to rounding."""
import numpy as np
import pytest

import workloads as wl
from oracle import dmrg as O
from oracle import grad as G
from tests import _layout as LY


def _case(kind, m, seed):
    rng = np.random.default_rng(seed)
    if kind == "chain":
        mpo, j = wl.heisenberg_chain(12), 5
    elif kind == "cyl":
        mpo, j = wl.heisenberg_square_cylinder(4, 3), 5
    else:
        mpo, j = wl.tfim_chain(10, 1.0, 0.7), 4
    qn = list(mpo.site.qn)
    bonds = wl.bond_sectors(mpo.L, qn, 0, m, sigma=None if kind == "tfim" else 3.0)
    bl, br = bonds[j], bonds[j + 2]
    W1, W2 = mpo.W[j], mpo.W[j + 1]
    f0, f2 = mpo.flux[j], mpo.flux[j + 2]
    Lenv = LY.random_env(bl, f0, rng)
    Renv = LY.random_env(br, f2, rng)
    keys = LY.psi_keys(bl, br, qn)
    psi = {k: rng.standard_normal((bl[k[0]], br[k[0] + qn[k[1]] + qn[k[2]]])) for k in keys}
    ybar = {k: rng.standard_normal(v.shape) for k, v in psi.items()}
    return rng, qn, Lenv, W1, f0, W2, f2, Renv, psi, ybar


def _phi(Lenv, W1, f0, W2, f2, Renv, psi, ybar, qn):
    y = O.heff_apply(Lenv, W1, f0, W2, f2, Renv, psi, qn)
    return sum(float(np.sum(ybar[k] * y[k])) for k in y)


def _dot(a, b):
    return sum(float(np.sum(a[k] * b[k])) for k in a)


def _shift(a, da, eps):
    return {k: a[k] + eps * da[k] for k in a}


@pytest.mark.parametrize("kind,m,seed", [("chain", 12, 1), ("cyl", 16, 2), ("tfim", 10, 3)])
def test_heff_gradients_match_finite_differences(kind, m, seed):
    rng, qn, Lenv, W1, f0, W2, f2, Renv, psi, ybar = _case(kind, m, seed)
    xbar, Lbar, Rbar, W1bar, W2bar = G.heff_backward(Lenv, W1, f0, W2, f2, Renv, psi, ybar, qn)
    eps = 1e-3
    phi = lambda L_=Lenv, W1_=W1, W2_=W2, R_=Renv, x_=psi: _phi(L_, W1_, f0, W2_, f2, R_, x_, ybar, qn)
    scale = abs(phi()) + 1.0
    # x
    dx = {k: rng.standard_normal(v.shape) for k, v in psi.items()}
    fd = (phi(x_=_shift(psi, dx, eps)) - phi(x_=_shift(psi, dx, -eps))) / (2 * eps)
    assert abs(fd - _dot(xbar, dx)) <= 1e-9 * scale
    # L and R
    dL = {k: rng.standard_normal(v.shape) for k, v in Lenv.items()}
    fd = (phi(L_=_shift(Lenv, dL, eps)) - phi(L_=_shift(Lenv, dL, -eps))) / (2 * eps)
    assert abs(fd - _dot(Lbar, dL)) <= 1e-9 * scale
    dR = {k: rng.standard_normal(v.shape) for k, v in Renv.items()}
    fd = (phi(R_=_shift(Renv, dR, eps)) - phi(R_=_shift(Renv, dR, -eps))) / (2 * eps)
    assert abs(fd - _dot(Rbar, dR)) <= 1e-9 * scale
    # MPO tensors: directions on the nonzero entries (the sparsity pattern is fixed)
    for W, Wbar, which in ((W1, W1bar, 1), (W2, W2bar, 2)):
        dW = np.where(W != 0.0, rng.standard_normal(W.shape), 0.0)
        if which == 1:
            fd = (phi(W1_=W1 + eps * dW) - phi(W1_=W1 - eps * dW)) / (2 * eps)
        else:
            fd = (phi(W2_=W2 + eps * dW) - phi(W2_=W2 - eps * dW)) / (2 * eps)
        assert abs(fd - float(np.sum(Wbar * dW))) <= 1e-9 * scale, which
        assert np.all(Wbar[W == 0.0] == 0.0)


def test_heff_gradient_of_the_local_energy_is_twice_the_matvec():
    """For a symmetric projected Hamiltonian (symmetric environments of a Hermitian MPO) the
    gradient of <x, H x> in x is 2 H x: with ybar = x, xbar = H^T x = H x."""
    mpo = wl.heisenberg_chain(10)
    qn = list(mpo.site.qn)
    j = 4
    bonds = wl.bond_sectors(mpo.L, qn, 0, 8, sigma=3.0)
    rng = np.random.default_rng(5)
    mps = wl.random_mps(mpo.L, qn, 0, 8, seed=4)
    st = O.SerialDMRG(mpo, mps)
    for jj in range(j):
        st.bond_step(jj, "right", 8)
    Lenv, Renv = st.Lenv[j], st.Renv[j + 2]
    psi = O.two_site(st.sites[j], st.sites[j + 1], qn)
    W1, W2, f0, f2 = mpo.W[j], mpo.W[j + 1], mpo.flux[j], mpo.flux[j + 2]
    y = O.heff_apply(Lenv, W1, f0, W2, f2, Renv, psi, qn)
    xbar = G.heff_backward(Lenv, W1, f0, W2, f2, Renv, psi, psi, qn)[0]
    for k in psi:
        assert np.abs(xbar[k] - y[k]).max() <= 1e-12 * (1 + np.abs(y[k]).max())
