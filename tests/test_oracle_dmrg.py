"""Pins for the oracle's serial two-site DMRG (Sec. II) against ED, closed forms,
library routines and invariants."""
import json
import os

import numpy as np
import pytest

import workloads as wl
from oracle import dmrg as D
from oracle import exact
from tests import _helpers as H

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "ed_energies.json")))


def _move_oc(eng, j):
    """Move the centre from site 0 to site j by untruncated SVDs."""
    qn = eng.qn
    m = eng.mpo
    for k in range(j):
        psi = D.two_site(eng.sites[k], eng.sites[k + 1], qn)
        A, lam, B, counts, _ = D.split_two_site(psi, eng.bonds[k], eng.bonds[k + 2], qn, 10 ** 9)
        eng.bonds[k + 1] = counts
        eng.sites[k] = A
        eng.sites[k + 1] = {(q, s): lam[q][:, None] * b for (q, s), b in B.items()}
        eng.Lenv[k + 1] = D.env_left(eng.Lenv[k], A, m.W[k], m.flux[k], m.flux[k + 1], qn)
    eng.oc = j


@pytest.mark.parametrize("model", ["heis", "tfim", "aklt", "cyl"])
def test_heff_matrix_equals_projected_global_hamiltonian(model):
    """Every element of the projected two-site Hamiltonian (built from L, W_i, W_{i+1}, R)
    equals E^T H E, with H the Kronecker-sum Hamiltonian and E the embedding of the bond's
    basis |a>|s1>|s2>|c> into the full space."""
    if model == "heis":
        L, site, terms, j = 7, wl.spin_half(), wl.heisenberg_terms(wl.chain_bonds(7)), 3
    elif model == "tfim":
        L, site, terms, j = 6, wl.spin_half_pauli(), wl.tfim_terms(6, 0.9, 1.2), 2
    elif model == "aklt":
        L, site, terms, j = 5, wl.spin_one(), wl.aklt_terms(5), 1
    else:
        L, site, terms, j = 8, wl.spin_half(), wl.heisenberg_terms(wl.square_cylinder_bonds(2, 4)), 4
    qtot = 1 if (model == "heis") else 0
    mpo = wl.build_mpo(L, site, terms, qtot=qtot)
    mps = wl.random_mps(L, site.qn, qtot, 6, seed=11)
    eng = D.SerialDMRG(mpo, mps)
    _move_oc(eng, j)
    qn = eng.qn
    psi = D.two_site(eng.sites[j], eng.sites[j + 1], qn)
    n = D.vflat(psi).size
    Hfull = exact.hamiltonian_sparse(L, site, terms).toarray()
    E = np.zeros((Hfull.shape[0], n))
    Heff = np.zeros((n, n))
    ops = eng.local_ops(j)
    for i in range(n):
        e = np.zeros(n)
        e[i] = 1.0
        blk = D.vunflat(e, psi)
        E[:, i] = H.embed_two_site(eng.sites, eng.bonds, j, blk, qn)
        Heff[:, i] = D.vflat(D.heff_apply(*ops, blk, qn))
    assert np.abs(E.T @ E - np.eye(n)).max() < 1e-12      # orthonormal basis (canonical form)
    assert np.abs(Heff - E.T @ Hfull @ E).max() < 1e-11
    dg = D.vflat(D.heff_diag(*ops, psi, qn))
    assert np.abs(dg - np.diag(Heff)).max() < 1e-12


def test_davidson_matches_dense_eigh():
    rng = np.random.default_rng(0)
    n = 300
    A = rng.standard_normal((n, n))
    A = A + A.T + np.diag(np.arange(n) * 0.5)
    ev = np.linalg.eigvalsh(A)[0]
    theta, u, it, rn = D.davidson(lambda x: A @ x, rng.standard_normal(n), np.diag(A).copy(), tol=1e-11, max_iter=500)
    assert abs(theta - ev) < 1e-9
    assert np.linalg.norm(A @ u - theta * u) < 1e-8


def test_truncation_rule():
    sv = {-2: np.array([0.5, 0.1]), 0: np.array([0.6, 0.3, 0.3 * (1 + 1e-12), 1e-15]), 2: np.array([0.5, 0.1])}
    # sorted: .6(0) .5(-2) .5(2) .3(0) .3(0) .1(-2) .1(2) -> m=4 cuts inside the .3 pair
    counts, err = D.truncate(sv, 4)
    assert counts == {-2: 1, 0: 1, 2: 1}
    counts, err = D.truncate(sv, 5)
    assert counts == {-2: 1, 0: 3, 2: 1}
    counts, _ = D.truncate(sv, 100)
    assert counts == {-2: 2, 0: 3, 2: 2}                   # 1e-15 below the 1e-12 relative cutoff
    tot = sum(float(np.sum(v * v)) for v in sv.values())
    _, err = D.truncate(sv, 3)
    assert abs(err - (2 * 0.09 + 2 * 0.01 + 1e-30) / tot) < 1e-12


def test_split_two_site_reconstructs_and_is_canonical():
    mps = wl.random_mps(6, (1, -1), 0, 8, seed=3)
    qn = [1, -1]
    psi = D.two_site(mps.sites[2], mps.sites[3], qn)
    A, lam, B, counts, err = D.split_two_site(psi, mps.bonds[2], mps.bonds[4], qn, 10 ** 9)
    assert err < 1e-28
    nrm = np.sqrt(D.vdot(psi, psi))
    rec = D.two_site({k: v * lam[k[0] + qn[k[1]]][None, :] for k, v in A.items()}, B, qn)
    for k in psi:
        assert np.abs(rec[k] * nrm - psi[k]).max() < 1e-12
    assert abs(sum(float(np.sum(v * v)) for v in lam.values()) - 1.0) < 1e-14
    for qm in counts:
        Ab = np.concatenate([A[(qa, s)] for (qa, s) in A if qa + qn[s] == qm], axis=0)
        Bb = np.concatenate([B[(q, s)] for (q, s) in B if q == qm], axis=1)
        assert np.abs(Ab.T @ Ab - np.eye(counts[qm])).max() < 1e-13
        assert np.abs(Bb @ Bb.T - np.eye(counts[qm])).max() < 1e-13


def test_right_canonical_start():
    mps = wl.random_mps(10, (1, -1), 0, 12, seed=4)
    sites, bonds = D.right_canonicalize(mps.sites, mps.bonds, [1, -1])
    v0 = H.mps_to_vector(mps.sites, mps.bonds, [1, -1])
    v1 = H.mps_to_vector(sites, bonds, [1, -1])
    assert abs(abs(v0 @ v1) / np.linalg.norm(v0) - 1.0) < 1e-12   # same state, normalised
    for j in range(1, 10):
        Rm = H.right_matrix(sites, bonds, j, [1, -1])
        assert np.abs(Rm @ Rm.T - np.eye(Rm.shape[0])).max() < 1e-12


def test_heisenberg_L16_exact_at_m256():
    L = 16
    mpo = wl.heisenberg_chain(L)
    eng = D.SerialDMRG(mpo, wl.random_mps(L, mpo.site.qn, 0, 16, seed=0))
    for _ in range(3):
        r = eng.sweep(256)
    assert abs(r["energy"] - GOLD["heisenberg_chain_L16_Sz0"]) < 1e-10


def test_heisenberg_L16_m64_variational():
    """Small config: 6 sweeps, m <= 64, random normal start (seed 0)."""
    L = 16
    mpo = wl.heisenberg_chain(L)
    eng = D.SerialDMRG(mpo, wl.random_mps(L, mpo.site.qn, 0, 64, seed=0))
    es = []
    for _ in range(6):
        r = eng.sweep(64)
        es.append(r["energy"])
    e0 = GOLD["heisenberg_chain_L16_Sz0"]
    assert es[-1] >= e0 - 1e-12
    assert es[-1] - e0 < 1e-8 * abs(e0)
    # energies at fixed m do not go up (beyond the truncation noise)
    for a, b in zip(es[1:], es[2:]):
        assert b <= a + 1e-11


def test_monotone_bond_energies_without_truncation():
    L = 10
    mpo = wl.heisenberg_chain(L)
    eng = D.SerialDMRG(mpo, wl.random_mps(L, mpo.site.qn, 0, 4, seed=2))
    r = eng.sweep(10 ** 6)
    e = [s["energy"] for s in r["steps"]]
    assert all(s["trunc"] < 1e-20 for s in r["steps"][1:])
    for a, b in zip(e, e[1:]):
        assert b <= a + 1e-12


@pytest.mark.parametrize("h", [0.5, 1.0, 1.5])
def test_tfim_closed_form(h):
    L = 32
    mpo = wl.tfim_chain(L, 1.0, h)
    eng = D.SerialDMRG(mpo, wl.random_mps(L, mpo.site.qn, 0, 8, seed=0))
    for _ in range(4):
        r = eng.sweep(24)
    e0 = exact.tfim_energy(L, 1.0, h)
    assert r["energy"] >= e0 - 1e-10
    assert abs(r["energy"] - e0) < 1e-8 * abs(e0)


def test_aklt_exact_at_small_m():
    L = 20
    mpo = wl.aklt_chain(L)
    eng = D.SerialDMRG(mpo, wl.random_mps(L, mpo.site.qn, 0, 8, seed=0))
    for _ in range(4):
        r = eng.sweep(8)
    assert abs(r["energy"] - exact.aklt_energy(L)) < 1e-10


def test_spin1_and_cylinders_against_ed():
    cases = [
        (wl.heisenberg_chain(10, spin="one"), "spin1_heisenberg_chain_L10_Sz0", 200),
        (wl.heisenberg_square_cylinder(4, 3), "heisenberg_cylinder_4x3_Sz0", 100),
        (wl.heisenberg_triangular_cylinder(4, 3), "heisenberg_triangular_4x3_Sz0", 100),
    ]
    for mpo, key, m in cases:
        eng = D.SerialDMRG(mpo, wl.random_mps(mpo.L, mpo.site.qn, 0, 16, seed=1))
        for _ in range(4):
            r = eng.sweep(m)
        assert abs(r["energy"] - GOLD[key]) < 1e-9, key


def test_sweep_energy_equals_global_expectation():
    L = 10
    mpo = wl.heisenberg_chain(L)
    eng = D.SerialDMRG(mpo, wl.random_mps(L, mpo.site.qn, 0, 8, seed=7))
    eng.sweep(6)
    v = H.mps_to_vector(eng.sites, eng.bonds, eng.qn)
    idx = exact.sector_states(L, eng.qn, 0)
    Hs = exact.hamiltonian_sparse(L, mpo.site, wl.heisenberg_terms(wl.chain_bonds(L)))
    e_full = (v @ (Hs @ v)) / (v @ v)
    assert np.abs(np.delete(v, idx)).max() == 0.0
    psi = D.two_site(eng.sites[0], eng.sites[1], eng.qn)
    assert abs(eng.energy_of(0, psi) - e_full) < 1e-12


def test_thin_svd_fallback_driver(monkeypatch):
    """thin_svd: the SVD of a graded matrix (reconstruction, orthonormal factors, descending
    values equal to the singular values from the eigenvalues of M^T M); the same when the
    divide-and-conquer driver reports non-convergence and the QR-iteration driver takes over; a
    non-finite entry raises instead of being retried."""
    rng = np.random.default_rng(9)
    M = rng.standard_normal((40, 25)) * np.logspace(0, -8, 25)[None, :]
    ref = np.sqrt(np.sort(np.linalg.eigvalsh(M.T @ M))[::-1].clip(0))

    def check(U, S, Vt):
        assert U.shape == (40, 25) and Vt.shape == (25, 25)
        assert np.all(np.diff(S) <= 0)
        assert np.abs((U * S) @ Vt - M).max() <= 1e-13
        assert np.abs(U.T @ U - np.eye(25)).max() <= 1e-13
        assert np.abs(Vt @ Vt.T - np.eye(25)).max() <= 1e-13
        assert np.abs(S[:8] - ref[:8]).max() <= 1e-12 * S[0]   # the well-resolved top of the spectrum

    check(*D.thin_svd(M))

    def fail(*a, **k):
        raise np.linalg.LinAlgError("SVD did not converge")

    monkeypatch.setattr(np.linalg, "svd", fail)
    check(*D.thin_svd(M))
    bad = M.copy()
    bad[3, 4] = np.nan
    with pytest.raises(FloatingPointError):
        D.thin_svd(bad)
