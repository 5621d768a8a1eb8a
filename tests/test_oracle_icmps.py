"""Pins for the oracle's inverse canonical gauge and local expectation values (Sec. IV) against
dense state vectors, Schmidt values from numpy's SVD, and closed forms."""
import json
import os

import numpy as np
import pytest

import workloads as wl
from oracle import dmrg as D
from oracle import exact
from oracle import icmps as IC
from tests import _helpers as H

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "ed_energies.json")))


def _absorb_right(psi, V, qn):
    """Site tensors psi_j V_{j+1} (V absorbed into the right index; the last site unchanged)."""
    out = []
    for j, s in enumerate(psi):
        v = V[j + 1]
        out.append(s if v is None else {(qa, t): b * v[qa + qn[t]][None, :] for (qa, t), b in s.items()})
    return out


def _absorb_left(psi, V):
    """Site tensors V_j psi_j (V absorbed into the left index; the first site unchanged)."""
    return [s if V[j] is None else {(qa, t): V[j][qa][:, None] * b for (qa, t), b in s.items()}
            for j, s in enumerate(psi)]


def _dense_one(v, L, d, j, op):
    T = v.reshape(d ** j, d, d ** (L - j - 1))
    return float(np.einsum("asb,st,atb->", T, op, T))


def _dense_two(v, L, d, j, op2):
    T = v.reshape(d ** j, d * d, d ** (L - j - 2))
    return float(np.einsum("asb,st,atb->", T, op2, T))


def _state(kind, L, m, seed):
    if kind == "half":
        site = wl.spin_half()
    else:
        site = wl.spin_one()
    qn = list(site.qn)
    qtot = (1 if L % 2 else 2) if kind == "half" else 0
    return site, qn, qtot, wl.random_mps(L, qn, qtot, m, seed=seed)


CASES = [("half", 9, 6, 1), ("half", 8, 16, 2), ("one", 6, 7, 3)]


@pytest.mark.parametrize("kind,L,m,seed", CASES)
def test_gauge_keeps_the_state_and_lambda_are_schmidt_values(kind, L, m, seed):
    site, qn, qtot, mps = _state(kind, L, m, seed)
    v0 = H.mps_to_vector(mps.sites, mps.bonds, qn)
    v0 /= np.linalg.norm(v0)
    psi, V, bonds = IC.inverse_canonical(mps.sites, mps.bonds, qn)
    v = H.mps_to_vector(_absorb_right(psi, V, qn), bonds, qn)
    assert np.abs(v - v0).max() < 1e-12
    d = len(qn)
    for b in range(1, L):
        S = np.linalg.svd(v0.reshape(d ** b, d ** (L - b)), compute_uv=False)
        S = S[S > 1e-12 * S[0]]
        lam = np.sort(np.concatenate([1.0 / x for x in V[b].values()]))[::-1]
        assert lam.shape == S.shape, b
        assert np.abs(lam - S).max() < 1e-12, b
        # sectors sorted descending, sizes match the bond
        for q, x in V[b].items():
            assert len(x) == bonds[b][q] and np.all(np.diff(x) >= 0)


@pytest.mark.parametrize("kind,L,m,seed", CASES)
def test_every_site_is_an_orthogonality_centre(kind, L, m, seed):
    site, qn, qtot, mps = _state(kind, L, m, seed)
    psi, V, bonds = IC.inverse_canonical(mps.sites, mps.bonds, qn)
    left = _absorb_right(psi, V, qn)
    right = _absorb_left(psi, V)
    for j in range(L):
        Lm = H.left_matrix(left, bonds, j, qn)            # sites 0..j-1, each times V on its right
        assert np.abs(Lm.T @ Lm - np.eye(Lm.shape[1])).max() < 1e-12, j
        Rm = H.right_matrix(right, bonds, j + 1, qn)      # V times sites j+1..L-1
        assert np.abs(Rm @ Rm.T - np.eye(Rm.shape[0])).max() < 1e-12, j
        # hence psi_j carries the Schmidt weights of both its bonds
        T = H.dense_site(psi[j], bonds[j], bonds[j + 1], qn)
        nl, nr = T.shape[0], T.shape[2]
        M = T.reshape(nl, -1)
        lam_l = np.ones(1) if V[j] is None else np.concatenate([1.0 / V[j][q] for q in bonds[j]])
        assert np.abs(M @ M.T - np.diag(lam_l ** 2)).max() < 1e-12
        M = T.transpose(2, 0, 1).reshape(nr, -1)
        lam_r = np.ones(1) if V[j + 1] is None else np.concatenate([1.0 / V[j + 1][q] for q in bonds[j + 1]])
        assert np.abs(M @ M.T - np.diag(lam_r ** 2)).max() < 1e-12


def _ops(site):
    d = site.d
    I = np.eye(d)
    ops1 = [site.op("Sz"), site.op("Sz*Sz"), site.op("Sp") + site.op("Sm"), np.diag(np.arange(1.0, d + 1))]
    sdot = np.kron(site.op("Sz"), site.op("Sz")) + 0.5 * (np.kron(site.op("Sp"), site.op("Sm"))
                                                          + np.kron(site.op("Sm"), site.op("Sp")))
    ops2 = [sdot, np.kron(site.op("Sz"), I), np.kron(I, site.op("Sz")), np.kron(site.op("Sp"), site.op("Sm"))]
    return ops1, ops2


@pytest.mark.parametrize("kind,L,m,seed", CASES)
def test_local_expectations_equal_dense(kind, L, m, seed):
    site, qn, qtot, mps = _state(kind, L, m, seed)
    v = H.mps_to_vector(mps.sites, mps.bonds, qn)
    v /= np.linalg.norm(v)
    psi, V, bonds = IC.inverse_canonical(mps.sites, mps.bonds, qn)
    ops1, ops2 = _ops(site)
    e1, e2 = IC.all_expectations(psi, V, qn, ops1, ops2)
    d = len(qn)
    for o, op in enumerate(ops1):
        for j in range(L):
            assert abs(e1[o, j] - _dense_one(v, L, d, j, op)) < 1e-12, (o, j)
    for o, op in enumerate(ops2):
        for j in range(L - 1):
            assert abs(e2[o, j] - _dense_two(v, L, d, j, op)) < 1e-12, (o, j)
    # S^z sum rule of the charge sector (charges are 2 S^z) and no S^x in a U(1) eigenstate
    assert abs(e1[0].sum() - qtot / 2) < 1e-12
    assert np.abs(e1[2]).max() < 1e-14
    # Sz x 1 on bond j and 1 x Sz on bond j - 1 both measure <Sz_j>
    assert np.abs(e2[1] - e1[0][:-1]).max() < 1e-12
    assert np.abs(e2[2] - e1[0][1:]).max() < 1e-12


def test_heisenberg_bond_energies_add_up_to_ed():
    """Converged L = 12 chain (exact at m = 64): the nearest-neighbour S.S values add up to the
    exact-diagonalisation ground-state energy."""
    L = 12
    mpo = wl.heisenberg_chain(L)
    eng = D.SerialDMRG(mpo, wl.random_mps(L, mpo.site.qn, 0, 16, seed=0))
    for _ in range(3):
        eng.sweep(64)
    psi, V, bonds = IC.inverse_canonical(eng.sites, eng.bonds, eng.qn)
    _, ops2 = _ops(mpo.site)
    _, e2 = IC.all_expectations(psi, V, eng.qn, (), ops2[:1])
    assert abs(e2[0].sum() - GOLD["heisenberg_chain_L12_Sz0"]) < 1e-10
    # reflection symmetry of the open chain
    assert np.abs(e2[0] - e2[0][::-1]).max() < 1e-8


def test_aklt_every_bond_at_minus_two_thirds():
    """AKLT chain: h_j = S.S + (S.S)^2/3 = 2 P_2 - 2/3 and every ground state is annihilated by
    every spin-2 projector P_2, so each bond's expectation value is exactly -2/3."""
    L = 14
    mpo = wl.aklt_chain(L)
    eng = D.SerialDMRG(mpo, wl.random_mps(L, mpo.site.qn, 0, 8, seed=0))
    for _ in range(4):
        eng.sweep(8)
    psi, V, bonds = IC.inverse_canonical(eng.sites, eng.bonds, eng.qn)
    _, ops2 = _ops(mpo.site)
    sdot = ops2[0]
    _, e2 = IC.all_expectations(psi, V, eng.qn, (), [sdot + sdot @ sdot / 3.0])
    assert np.abs(e2[0] + 2.0 / 3.0).max() < 1e-10


def test_tfim_transverse_magnetisation_is_minus_dE_dh():
    """TFIM (no U(1) labels): sum_j <sigma^x_j> = -dE/dh (Hellmann-Feynman) of the free-fermion
    closed form, and sum_j <sigma^z_j sigma^z_{j+1}> = -dE/dJ."""
    L, J, h = 16, 1.0, 0.8
    mpo = wl.tfim_chain(L, J, h)
    eng = D.SerialDMRG(mpo, wl.random_mps(L, mpo.site.qn, 0, 8, seed=0))
    for m in (16, 32, 32, 32):
        eng.sweep(m)
    psi, V, bonds = IC.inverse_canonical(eng.sites, eng.bonds, eng.qn)
    X, Z = mpo.site.op("X"), mpo.site.op("Z")
    e1, e2 = IC.all_expectations(psi, V, eng.qn, [X], [np.kron(Z, Z)])
    st = 1e-5
    dEdh = (exact.tfim_energy(L, J, h + st) - exact.tfim_energy(L, J, h - st)) / (2 * st)
    dEdJ = (exact.tfim_energy(L, J + st, h) - exact.tfim_energy(L, J - st, h)) / (2 * st)
    assert abs(e1[0].sum() + dEdh) < 1e-7 * abs(dEdh)
    assert abs(e2[0].sum() + dEdJ) < 1e-7 * abs(dEdJ)


def test_a_dropped_v_is_detected():
    """Planted mistake: Theta = psi_j psi_{j+1} without V gives wrong bond values."""
    site, qn, qtot, mps = _state("half", 8, 8, 4)
    v = H.mps_to_vector(mps.sites, mps.bonds, qn)
    v /= np.linalg.norm(v)
    psi, V, bonds = IC.inverse_canonical(mps.sites, mps.bonds, qn)
    ones = [None if x is None else {q: np.ones_like(a) for q, a in x.items()} for x in V]
    _, ops2 = _ops(site)
    _, good = IC.all_expectations(psi, V, qn, (), ops2[:1])
    _, bad = IC.all_expectations(psi, ones, qn, (), ops2[:1])
    ref = np.array([_dense_two(v, 8, 2, j, ops2[0]) for j in range(7)])
    assert np.abs(good[0] - ref).max() < 1e-12
    assert np.abs(bad[0] - ref).max() > 1e-3
