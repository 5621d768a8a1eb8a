"""GPU two-site DMRG (FP64 mode, C ABI) against the CPU oracle: energies, block tables and
singular values sweep by sweep; closed-form pins; real-space regions."""
import json
import os

import numpy as np
import pytest

import workloads as wl
from oracle import dmrg as O
from oracle import exact
from oracle import regions as P
from tests._gpu import engine_for, load_mps

pytestmark = pytest.mark.gpu
pd = pytest.importorskip("paper_1301_3494_gb300")
GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "ed_energies.json")))
TOL = 1e-8     # FP64 parity: |dE/E|


def test_initial_energy_matches_oracle():
    L = 10
    mpo = wl.heisenberg_chain(L)
    mps = wl.random_mps(L, mpo.site.qn, 0, 12, seed=5)
    ref = O.SerialDMRG(mpo, mps)
    e_ref = ref.energy_of(0, O.two_site(ref.sites[0], ref.sites[1], ref.qn))
    eng = engine_for(pd, mpo)
    load_mps(eng, mps, ref.qn)
    e = eng.energy()
    assert abs(e - e_ref) <= 1e-12 * abs(e_ref)
    for b in range(L + 1):
        assert eng.bond(b) == ref.bonds[b]


def test_heisenberg_L16_m64_six_sweeps_parity():
    """Small config: L=16, D=5, m <= 64, 6 sweeps, random normal start (seed 0)."""
    L = 16
    mpo = wl.heisenberg_chain(L)
    mps = wl.random_mps(L, mpo.site.qn, 0, 64, seed=0)
    ref = O.SerialDMRG(mpo, mps)
    eng = engine_for(pd, mpo)
    load_mps(eng, mps, ref.qn)
    for sweep in range(6):
        r = ref.sweep(64)
        g = eng.sweep(64, dav_tol=1e-10, dav_max_iter=100)
        assert abs(g["energy"] - r["energy"]) <= TOL * abs(r["energy"]), sweep
        for b in range(L + 1):
            assert eng.bond(b) == ref.bonds[b], (sweep, b)
    e0 = GOLD["heisenberg_chain_L16_Sz0"]
    assert g["energy"] >= e0 - 1e-10
    assert g["energy"] - e0 < 1e-8 * abs(e0)
    # singular values at the centre bond
    lam = eng.lam(8)
    lr = np.concatenate([ref.lam[8][q] for q in sorted(ref.lam[8])])
    assert np.abs(np.sort(lam) - np.sort(lr)).max() < 1e-8


@pytest.mark.parametrize("h", [0.5, 1.0, 1.5])
def test_tfim_closed_form(h):
    L = 32
    mpo = wl.tfim_chain(L, 1.0, h)
    eng = engine_for(pd, mpo)
    load_mps(eng, wl.random_mps(L, mpo.site.qn, 0, 8, seed=0), list(mpo.site.qn))
    for _ in range(4):
        g = eng.sweep(24)
    e0 = exact.tfim_energy(L, 1.0, h)
    assert g["energy"] >= e0 - 1e-10
    assert abs(g["energy"] - e0) < 1e-8 * abs(e0)


def test_aklt_exact():
    L = 20
    mpo = wl.aklt_chain(L)
    eng = engine_for(pd, mpo)
    load_mps(eng, wl.random_mps(L, mpo.site.qn, 0, 8, seed=0), list(mpo.site.qn))
    for _ in range(4):
        g = eng.sweep(8)
    assert abs(g["energy"] - exact.aklt_energy(L)) < 1e-10


def test_cylinder_against_ed():
    mpo = wl.heisenberg_square_cylinder(4, 3)
    eng = engine_for(pd, mpo)
    load_mps(eng, wl.random_mps(mpo.L, mpo.site.qn, 0, 64, seed=1), list(mpo.site.qn))
    for _ in range(4):
        g = eng.sweep(100)
    assert abs(g["energy"] - GOLD["heisenberg_cylinder_4x3_Sz0"]) < 1e-9


@pytest.mark.parametrize("R,warm", [(2, 1), (4, 0)])
def test_regions_match_oracle(R, warm):
    L = 16
    mpo = wl.heisenberg_chain(L)
    mps = wl.random_mps(L, mpo.site.qn, 0, 8, seed=0)
    ref = P.ParallelDMRG(mpo, mps, R)
    ref.setup(32, warmup_sweeps=warm)
    eng = engine_for(pd, mpo)
    load_mps(eng, mps, list(mpo.site.qn))
    eng.setup_regions(R, warm, 32)
    for k in range(R):
        assert eng.center(k) == ref.regions[k].oc
    for sweep, m in enumerate((32, 64, 64)):
        r = ref.sweep(m)
        g = eng.sweep(m)
        assert abs(g["energy"] - r["energy"]) <= TOL * abs(r["energy"]), sweep
        fids = [x["fidelity"] for x in r["merges"]]
        assert abs(g["max_fidelity"] - max(fids)) <= 1e-7
    assert abs(g["energy"] - GOLD["heisenberg_chain_L16_Sz0"]) < 1e-7


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
def test_mixed_precision_energy_within_1e5(prec):
    """Mixed precision (tensor-core matvec and environments, FP32 SVD on ordinary bonds, FP64
    Davidson small problem and orthogonalisation): the converged energy, evaluated as an FP64
    Rayleigh quotient, agrees with the FP64 oracle to 1e-5 relative."""
    L = 30
    mpo = wl.heisenberg_chain(L)
    mps = wl.random_mps(L, mpo.site.qn, 0, 16, seed=0)
    ref = O.SerialDMRG(mpo, mps)
    eng = engine_for(pd, mpo, precision=prec)
    load_mps(eng, mps, list(mpo.site.qn))
    for m in (32, 64, 64, 64):
        r = ref.sweep(m)
        # bf16 Ritz vectors start further from the accurate ones, so they get more refinement
        g = eng.sweep(m, dav_tol=1e-9, dav_max_iter=12, refine_iters=3 if prec == "tf32" else 6)
    e64 = eng.energy()
    assert abs(e64 - r["energy"]) <= 1e-5 * abs(r["energy"]), (e64, r["energy"])
    assert abs(g["energy"] - r["energy"]) <= 1e-4 * abs(r["energy"])


def test_mixed_precision_regions_within_1e5():
    """Real-space parallel sweeps in mixed precision: four regions run concurrently on their own
    streams (bf16 matvec, FP32 block-Jacobi SVD launched round by round, FP64 accurate SVD at the
    shared bonds).  The sweep energy agrees with the FP64 oracle's converged serial energy to 1e-5
    relative."""
    L = 32
    mpo = wl.heisenberg_chain(L)
    mps = wl.random_mps(L, mpo.site.qn, 0, 16, seed=0)
    ref = O.SerialDMRG(mpo, mps)
    for m in (32, 64, 64, 64):
        r = ref.sweep(m)
    eng = engine_for(pd, mpo, precision="bf16")
    load_mps(eng, mps, list(mpo.site.qn))
    eng.setup_regions(4, 1, 32, dav_tol=1e-9, dav_max_iter=12, refine_iters=6)
    for m in (32, 64, 64, 64, 64):
        g = eng.sweep(m, dav_tol=1e-9, dav_max_iter=12, refine_iters=6)
    assert abs(g["energy"] - r["energy"]) <= 1e-5 * abs(r["energy"]), (g["energy"], r["energy"])


def test_state_export_round_trip():
    """dmrg_get_site / dmrg_get_bond / dmrg_get_center reproduce the state through dmrg_set_mps:
    a second engine built from the export has the same FP64 energy and the same bond tables."""
    L = 16
    mpo = wl.heisenberg_chain(L)
    mps = wl.random_mps(L, mpo.site.qn, 0, 8, seed=3)
    eng = engine_for(pd, mpo)
    load_mps(eng, mps, list(mpo.site.qn))
    for m in (16, 32):
        eng.sweep(m)
    bonds, data, c = eng.state()
    e1 = eng.energy()
    eng2 = engine_for(pd, mpo)
    eng2.set_mps(bonds, data, center=c)
    assert abs(eng2.energy() - e1) <= 1e-12 * abs(e1)
    assert all(eng2.bond(b) == bonds[b] for b in range(L + 1))
    eng.close()
    eng2.close()


@pytest.mark.parametrize("schedule", [1, 2])
@pytest.mark.parametrize("R", [2, 4])
def test_regions_cylinder_serial_schedule(R, schedule):
    """6x4 Heisenberg cylinder with a random longitudinal field (2-D snake MPO, D = 14; the field
    lifts the SU(2) and spin-flip degeneracies of the Schmidt values, so the cut has no
    symmetry-enforced near-ties), m = 128 in the set-up and the sweeps, the regions of each Fig. 4
    phase driven by the calling thread -- one after another (serial_regions = 1, cooperative Jacobi
    launches inside the regions) or in lockstep, bond step by bond step (serial_regions = 2):
    region centres, sweep energies and merge fidelities match the
    FP64 oracle sweep by sweep, and so do the bond tables of every bond the truncation cuts at m
    (bonds kept whole end in singular values near the 1e-12 cutoff, whose vectors are not
    determined by the wavefunction)."""
    m = 128
    mpo = wl.field_square_cylinder(6, 4, seed=3)
    qn = list(mpo.site.qn)
    mps = wl.random_mps(mpo.L, qn, 0, 16, seed=2)
    ref = P.ParallelDMRG(mpo, mps, R)
    ref.setup(m, warmup_sweeps=1)
    eng = engine_for(pd, mpo)
    load_mps(eng, mps, qn)
    eng.setup_regions(R, 1, m, serial_regions=schedule)
    for k in range(R):
        assert eng.center(k) == ref.regions[k].oc
    for sweep in range(2):
        r = ref.sweep(m)
        g = eng.sweep(m, serial_regions=schedule)
        assert abs(g["energy"] - r["energy"]) <= TOL * abs(r["energy"]), sweep
        fids = [x["fidelity"] for x in r["merges"]]
        assert abs(g["max_fidelity"] - max(fids)) <= 1e-7 * max(1.0, max(fids)), (g["max_fidelity"], fids)
        assert abs(g["min_fidelity"] - min(fids)) <= 1e-7 * max(1.0, max(fids)), (g["min_fidelity"], fids)
    cut = 0
    for k, reg in enumerate(ref.regions):
        assert eng.center(k) == reg.oc
        for b in range(reg.p + 1, reg.q + 1):
            if sum(reg.bonds[b].values()) == m:
                cut += 1
                assert eng.bond(b) == reg.bonds[b], (k, b)
    assert cut >= 4
    eng.close()


def test_regions_cylinder_serial_schedule_bf16():
    """The bench's code path on a 2-D MPO: bf16 tensor-core matvec with FP32 refinement, FP32
    block-Jacobi splits (cooperative launch) on ordinary bonds, FP64 accurate splits and merges at
    the shared bonds, 4 regions on the serial schedule.  The final parallel-sweep energy agrees
    with the FP64 oracle's converged serial energy of the 6x4 field cylinder at m = 128 to 2e-5
    (FP32 environments bias the mixed engine's own Rayleigh quotient at the 1e-5 level)."""
    mpo = wl.field_square_cylinder(6, 4, seed=3)
    qn = list(mpo.site.qn)
    mps = wl.random_mps(mpo.L, qn, 0, 16, seed=2)
    ref = O.SerialDMRG(mpo, mps)
    for m in (64, 128, 128, 128):
        r = ref.sweep(m)
    eng = engine_for(pd, mpo, precision="bf16")
    load_mps(eng, mps, qn)
    dav = dict(dav_tol=1e-9, dav_max_iter=12, refine_iters=6, serial_regions=1)
    eng.setup_regions(4, 1, 128, **dav)
    for m in (128, 128, 128, 128):
        g = eng.sweep(m, **dav)
    assert abs(g["energy"] - r["energy"]) <= 2e-5 * abs(r["energy"]), (g["energy"], r["energy"])
    eng.close()


def test_regions_lockstep_bf16_matches_serial():
    """The bench's mixed-precision path with the regions in lockstep (serial_regions = 2: every
    Fig. 4 phase's FP32 splits of all regions in one grouped block-Jacobi launch) against the same
    engine with the regions one after another (serial_regions = 1) and the FP64 oracle's converged
    serial energy: the two schedules differ only by the rounding of the FP32 splits, so their
    sweep energies agree to 1e-5 (the mixed engine's own accuracy level on FP32 environments) and
    both reach the oracle's to 2e-5; the same bonds are split, in fewer split passes."""
    mpo = wl.field_square_cylinder(6, 4, seed=3)
    qn = list(mpo.site.qn)
    mps = wl.random_mps(mpo.L, qn, 0, 16, seed=2)
    ref = O.SerialDMRG(mpo, mps)
    for m in (64, 128, 128, 128):
        r = ref.sweep(m)
    out = []
    for schedule in (1, 2):
        eng = engine_for(pd, mpo, precision="bf16")
        load_mps(eng, mps, qn)
        dav = dict(dav_tol=1e-9, dav_max_iter=12, refine_iters=6, serial_regions=schedule)
        eng.setup_regions(4, 1, 96, **dav)
        pd.profile_enable(True)
        pd.profile_reset()
        gs = [eng.sweep(m, **dav) for m in (96, 128, 128, 128)]
        prof = pd.profile_read()
        pd.profile_enable(False)
        out.append((gs, [eng.bond(b) for b in range(mpo.L + 1)], prof))
        eng.close()
    (g1, b1, p1), (g2, b2, p2) = out
    for x, y in zip(g1, g2):
        assert abs(x["energy"] - y["energy"]) <= 1e-5 * abs(x["energy"]), (x["energy"], y["energy"])
    for g in (g1[-1], g2[-1]):
        assert abs(g["energy"] - r["energy"]) <= 2e-5 * abs(r["energy"]), (g["energy"], r["energy"])
    assert all(sum(x.values()) <= 128 for x in b2)
    # (an FP32 split refused by the FP64 re-orthonormalisation is redone alone in FP64)
    assert p1["svd_bonds"] - p1["svd_fp64_fallbacks"] == p2["svd_bonds"] - p2["svd_fp64_fallbacks"]
    assert p2["svd_calls"] < p2["svd_bonds"] / 2
    assert p1["svd_calls"] == p1["svd_bonds"]


def test_region_state_export():
    """The region state exported as one MPS (dmrg_get_site in region mode, V = Lambda^-1 of each
    boundary in the first site to its right) is the oracle's region state contracted with V at
    every boundary, Eq. (merge): same dense vector up to sign and norm; an FP64 engine that loads
    it (canonicalising it itself) reports its dense Rayleigh quotient."""
    from tests._helpers import mps_to_vector, mpo_to_matrix
    L, R = 12, 3
    mpo = wl.heisenberg_chain(L)
    qn = list(mpo.site.qn)
    mps = wl.random_mps(L, qn, 0, 8, seed=6)
    ref = P.ParallelDMRG(mpo, mps, R)
    ref.setup(16, warmup_sweeps=1)
    eng = engine_for(pd, mpo)
    load_mps(eng, mps, qn)
    eng.setup_regions(R, 1, 16)
    for _ in range(2):
        ref.sweep(16)
        eng.sweep(16)
    bonds, data = eng.region_state()
    sites, off = [], 0
    for j in range(L):
        n = sum(bonds[j][q] * bonds[j + 1][q + s] for q in bonds[j] for s in qn if q + s in bonds[j + 1])
        sites.append(wl.unpack_site(data[off: off + n], bonds[j], bonds[j + 1], qn))
        off += n
    v = mps_to_vector(sites, bonds, qn)
    # the oracle's region state, V inserted at the boundaries
    osites, obonds = [], [None] * (L + 1)
    for k, reg in enumerate(ref.regions):
        for b in range(reg.p, reg.q + 2):
            obonds[b] = reg.bonds[b]
        for j in range(reg.p, reg.q + 1):
            blk = reg.sites[j]
            if k > 0 and j == reg.p:
                V = ref.V[j]
                blk = {(ql, s): V[ql][:, None] * x for (ql, s), x in blk.items()}
            osites.append(blk)
    vo = mps_to_vector(osites, obonds, qn)
    ov = abs(v @ vo) / (np.linalg.norm(v) * np.linalg.norm(vo))
    assert 1.0 - ov <= 1e-9, ov
    H = mpo_to_matrix(mpo)
    e_dense = float(v @ H @ v / (v @ v))
    eng2 = engine_for(pd, mpo)
    eng2.set_mps(bonds, data)
    assert abs(eng2.energy() - e_dense) <= 1e-11 * abs(e_dense)
    eng.close()
    eng2.close()


def test_mixed_regions_fp64_edges_merge_predicts():
    """bf16 regions with FP64-accurate environments and FP64 solves next to the boundaries (the
    edge tensors psi_3, psi_4 of Eq. (merge) and the merges): the merge prediction
    Psi' = psi'_3 V psi'_4 stays a good initial guess (fidelity 1 - |<Psi'|Psi>| below 1e-2 once
    converged; the bf16-only solves leave it near 1), and the parallel-sweep energy -- a Rayleigh
    quotient on FP64-accurate environments -- agrees with the FP64 oracle to 1e-5."""
    L = 32
    mpo = wl.heisenberg_chain(L)
    qn = list(mpo.site.qn)
    mps = wl.random_mps(L, qn, 0, 16, seed=0)
    ref = O.SerialDMRG(mpo, mps)
    for m in (32, 64, 64, 64):
        r = ref.sweep(m)
    W, flux, D = wl.pack_mpo(mpo)
    eng = pd.Engine(W, flux, D, qn, 0, "bf16", 8, fp64_emulation=True, env_fp64=True, accurate_edges=True)
    load_mps(eng, mps, qn)
    dav = dict(dav_tol=1e-9, dav_max_iter=12, refine_iters=6, serial_regions=1)
    eng.setup_regions(4, 1, 32, **dav)
    for m in (32, 64, 64, 64, 64, 64):
        g = eng.sweep(m, **dav)
    assert g["max_fidelity"] <= 1e-2, g["max_fidelity"]
    assert abs(g["energy"] - r["energy"]) <= 1e-5 * abs(r["energy"]), (g["energy"], r["energy"])
    assert g["n_refine_matvec"] > 0
    eng.close()
