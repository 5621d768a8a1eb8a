"""Pins for the real-space parallel scheme (Sec. II, Eqs. inverse, isvd, merge; Fig. 4)."""
import json
import os

import numpy as np
import pytest

import workloads as wl
from oracle import dmrg as D
from oracle import regions as P

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "ed_energies.json")))


def test_isvd_identity():
    """Psi = psi_3 V psi_4 with psi_3 = A Lambda, psi_4 = Lambda B, V = Lambda^{-1} (Eq. isvd)."""
    mps = wl.random_mps(6, (1, -1), 0, 8, seed=3)
    qn = [1, -1]
    psi = D.two_site(mps.sites[2], mps.sites[3], qn)
    nrm = np.sqrt(D.vdot(psi, psi))
    A, lam, B, _, _ = D.split_two_site(psi, mps.bonds[2], mps.bonds[4], qn, 10 ** 9)
    psi3 = {k: v * lam[k[0] + qn[k[1]]][None, :] for k, v in A.items()}
    psi4 = {k: lam[k[0]][:, None] * v for k, v in B.items()}
    V = {q: 1.0 / v for q, v in lam.items()}
    rec = D.two_site({k: v * V[k[0] + qn[k[1]]][None, :] for k, v in psi3.items()}, psi4, qn)
    for k in psi:
        assert np.abs(rec[k] * nrm - psi[k]).max() < 1e-12


@pytest.mark.parametrize("R", [2, 4])
def test_exact_state_is_a_merge_fixed_point(R):
    """An untruncated converged state is a fixed point of the merge: fidelity 1 - |<Psi'|Psi>|
    is zero and the energy does not move."""
    L = 12
    mpo = wl.heisenberg_chain(L)
    par = P.ParallelDMRG(mpo, wl.random_mps(L, mpo.site.qn, 0, 16, seed=0), R)
    par.setup(4096, warmup_sweeps=3)
    r = par.sweep(4096)
    e0 = GOLD["heisenberg_chain_L12_Sz0"]
    for mg in r["merges"]:
        assert mg["fidelity"] < 1e-12
        assert abs(mg["energy"] - e0) < 1e-11


@pytest.mark.parametrize("R,warm", [(2, 0), (2, 1), (4, 0), (4, 2)])
def test_parallel_converges_to_ed(R, warm):
    L = 16
    mpo = wl.heisenberg_chain(L)
    par = P.ParallelDMRG(mpo, wl.random_mps(L, mpo.site.qn, 0, 8, seed=0), R)
    par.setup(32, warmup_sweeps=warm)
    for _ in range(4):
        r = par.sweep(256)
    assert abs(r["energy"] - GOLD["heisenberg_chain_L16_Sz0"]) < 1e-9


def test_staggered_positions_and_boundaries():
    L = 20
    mpo = wl.heisenberg_chain(L)
    par = P.ParallelDMRG(mpo, wl.random_mps(L, mpo.site.qn, 0, 8, seed=0), 4)
    assert par.bounds == [0, 5, 10, 15, 20]
    par.setup(16)
    # odd regions (1-based) sit at their left end, even ones at their right end
    assert [r.oc for r in par.regions] == [0, 9, 10, 19]
    r = par.sweep(16)
    assert [m["boundary"] for m in r["merges"]] == [5, 15, 10]
    assert [r.oc for r in par.regions] == [0, 9, 10, 19]


def test_merge_fidelity_is_small_but_nonzero_when_truncated():
    """Fig. 3's qualitative statement: the merged state is a good but not exact guess."""
    L = 24
    mpo = wl.heisenberg_chain(L)
    par = P.ParallelDMRG(mpo, wl.random_mps(L, mpo.site.qn, 0, 8, seed=0), 2)
    par.setup(8, warmup_sweeps=1)
    fids = []
    for m in (8, 16, 16, 24):
        r = par.sweep(m)
        fids.append(r["merges"][0]["fidelity"])
    assert 0.0 < fids[-1] < 1e-2
