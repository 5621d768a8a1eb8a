"""GPU inverse canonical gauge and local expectation values (Sec. IV) against the oracle on the
same exported state: bond sectors bit-exact, Schmidt values and expectation values within 1e-12,
every exported site tensor an orthogonality centre, closed-form sums on converged states."""
import numpy as np
import pytest

import workloads as wl
from oracle import exact as EX
from oracle import icmps as IC
from tests._gpu import engine_for, load_mps

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

pd = pytest.importorskip("paper_1301_3494_gb300")


def _oracle_state(eng, qn):
    bonds, data, _ = eng.state()
    sites, off = [], 0
    for j in range(eng.L):
        n = sum(bonds[j][q] * bonds[j + 1][q + s] for q in bonds[j] for s in qn if q + s in bonds[j + 1])
        sites.append(wl.unpack_site(data[off: off + n], bonds[j], bonds[j + 1], qn))
        off += n
    return sites, bonds


def _ops(site):
    d = site.d
    I = np.eye(d)
    if "Sz" in site.ops:
        Sz, Sp, Sm = site.op("Sz"), site.op("Sp"), site.op("Sm")
        ops1 = [Sz, Sz @ Sz, Sp + Sm, np.diag(np.arange(1.0, d + 1))]
        sdot = np.kron(Sz, Sz) + 0.5 * (np.kron(Sp, Sm) + np.kron(Sm, Sp))
        ops2 = [sdot, np.kron(Sz, I), np.kron(I, Sz), np.kron(Sp, Sm)]
    else:
        X, Z = site.op("X"), site.op("Z")
        ops1 = [X, Z, np.diag([1.0, 2.0])]
        ops2 = [np.kron(Z, Z), np.kron(X, I), np.kron(X, X)]
    return ops1, ops2


def _case(kind, m, seed, sweeps):
    if kind == "chain":
        mpo = wl.heisenberg_chain(20)
    elif kind == "spin1":
        mpo = wl.heisenberg_chain(12, spin="one")
    elif kind == "cyl":
        mpo = wl.heisenberg_square_cylinder(6, 4)
    elif kind == "tfim":
        mpo = wl.tfim_chain(18, 1.0, 0.9)
    else:                                   # long chain, blocks above one dot chunk
        mpo = wl.heisenberg_chain(24)
    qn = list(mpo.site.qn)
    eng = engine_for(pd, mpo)
    sigma = 1.5 if kind == "long" else None          # few large sectors: blocks above 32768 elements
    load_mps(eng, wl.random_mps(mpo.L, qn, mpo.qtot, m, seed=seed, sigma=sigma), qn)
    for _ in range(sweeps):
        eng.sweep(m)
    return mpo, qn, eng


def _unpack(eng, j, bonds, qn):
    return wl.unpack_site(eng.icmps_site(j), bonds[j], bonds[j + 1], qn)


@pytest.mark.parametrize("kind,m,seed,sweeps", [("chain", 24, 1, 0), ("chain", 32, 2, 2), ("spin1", 20, 3, 1),
                                                ("cyl", 90, 4, 0), ("tfim", 16, 5, 1), ("long", 600, 6, 0)])
def test_gauge_and_expectations_match_oracle(kind, m, seed, sweeps):
    mpo, qn, eng = _case(kind, m, seed, sweeps)
    sites, bonds0 = _oracle_state(eng, qn)
    psi_o, V_o, bonds_o = IC.inverse_canonical(sites, bonds0, qn)
    eng.inverse_canonical()
    L = mpo.L
    bonds = [eng.icmps_bond(b) for b in range(L + 1)]
    assert bonds == bonds_o                                    # sector structure bit-exact
    lam = [None] * (L + 1)
    for b in range(1, L):
        v = eng.icmps_v(b)
        off = 0
        lam[b] = {}
        for q, k in bonds[b].items():
            lam[b][q] = 1.0 / v[off: off + k]
            assert np.abs(lam[b][q] - 1.0 / V_o[b][q]).max() <= 1e-12, (b, q)
            off += k
    # every GPU site tensor is an orthogonality centre carrying the Schmidt weights of both bonds
    for j in range(L):
        blocks = _unpack(eng, j, bonds, qn)
        for q in bonds[j]:
            rows = [blk for (ql, s), blk in blocks.items() if ql == q]
            M = sum(b_ @ b_.T for b_ in rows)
            want = np.diag(lam[j][q] ** 2) if j > 0 else np.ones((1, 1))
            assert np.abs(M - want).max() <= 1e-12, (j, q)
        for q in bonds[j + 1]:
            cols = [blk for (ql, s), blk in blocks.items() if ql + qn[s] == q]
            M = sum(b_.T @ b_ for b_ in cols)
            want = np.diag(lam[j + 1][q] ** 2) if j + 1 < L else np.ones((1, 1))
            assert np.abs(M - want).max() <= 1e-12, (j, q)
    ops1, ops2 = _ops(mpo.site)
    e1_o, e2_o = IC.all_expectations(psi_o, V_o, qn, ops1, ops2)
    e1, e2, ms = eng.local_expectations(ops1, ops2)
    assert e1.shape == e1_o.shape and e2.shape == e2_o.shape
    assert np.abs(e1 - e1_o).max() <= 1e-12
    assert np.abs(e2 - e2_o).max() <= 1e-12
    assert ms > 0.0
    eng.close()


def test_converged_sums_against_closed_forms():
    """Heisenberg L = 20: the S.S bond values add up to the engine's energy; TFIM L = 16: the
    transverse magnetisation is -dE/dh of the free-fermion closed form."""
    mpo = wl.heisenberg_chain(20)
    qn = list(mpo.site.qn)
    eng = engine_for(pd, mpo)
    load_mps(eng, wl.random_mps(20, qn, 0, 16, seed=0), qn)
    for m in (32, 64, 96, 96):
        eng.sweep(m)
    e = eng.energy()
    eng.inverse_canonical()
    _, ops2 = _ops(mpo.site)
    e1, e2, _ = eng.local_expectations([mpo.site.op("Sz")], ops2[:1])
    assert abs(e2[0].sum() - e) <= 1e-10 * abs(e)
    assert abs(e1[0].sum()) <= 1e-12
    assert np.abs(e2[0] - e2[0][::-1]).max() <= 1e-5            # reflection symmetry (up to truncation)
    eng.close()
    L, J, h = 16, 1.0, 0.8
    mpo = wl.tfim_chain(L, J, h)
    eng = engine_for(pd, mpo)
    load_mps(eng, wl.random_mps(L, mpo.site.qn, 0, 8, seed=0), list(mpo.site.qn))
    for m in (16, 32, 32, 32):
        eng.sweep(m)
    eng.inverse_canonical()
    e1, e2, _ = eng.local_expectations([mpo.site.op("X")], [np.kron(mpo.site.op("Z"), mpo.site.op("Z"))])
    st = 1e-5
    dEdh = (EX.tfim_energy(L, J, h + st) - EX.tfim_energy(L, J, h - st)) / (2 * st)
    dEdJ = (EX.tfim_energy(L, J + st, h) - EX.tfim_energy(L, J - st, h)) / (2 * st)
    assert abs(e1[0].sum() + dEdh) <= 1e-7 * abs(dEdh)
    assert abs(e2[0].sum() + dEdJ) <= 1e-7 * abs(dEdJ)
    eng.close()


def test_mixed_precision_state_gauged_in_fp64():
    """A bf16 engine's state: the gauge and the measurement run in FP64 on its site tensors, so
    they agree with the oracle on the exported state to FP64 accuracy."""
    mpo = wl.heisenberg_square_cylinder(6, 4)
    qn = list(mpo.site.qn)
    eng = engine_for(pd, mpo, precision="bf16")
    load_mps(eng, wl.random_mps(mpo.L, qn, 0, 32, seed=8), qn)
    for _ in range(2):
        eng.sweep(64)
    sites, bonds0 = _oracle_state(eng, qn)
    psi_o, V_o, _ = IC.inverse_canonical(sites, bonds0, qn)
    eng.inverse_canonical()
    ops1, ops2 = _ops(mpo.site)
    e1_o, e2_o = IC.all_expectations(psi_o, V_o, qn, ops1, ops2)
    e1, e2, _ = eng.local_expectations(ops1, ops2)
    assert np.abs(e1 - e1_o).max() <= 1e-11
    assert np.abs(e2 - e2_o).max() <= 1e-11
    eng.close()


def test_copy_is_discarded_when_the_state_changes():
    mpo = wl.heisenberg_chain(10)
    qn = list(mpo.site.qn)
    eng = engine_for(pd, mpo)
    load_mps(eng, wl.random_mps(10, qn, 0, 8, seed=1), qn)
    with pytest.raises(pd.DMRGError) as ex:
        eng.local_expectations([mpo.site.op("Sz")])
    assert ex.value.status == 8
    eng.inverse_canonical()
    e1, _, _ = eng.local_expectations([mpo.site.op("Sz")])
    assert abs(e1.sum()) <= 1e-12
    eng.sweep(8)
    with pytest.raises(pd.DMRGError) as ex:
        eng.local_expectations([mpo.site.op("Sz")])
    assert ex.value.status == 8
    # empty operator lists are valid
    eng.inverse_canonical()
    e1, e2, _ = eng.local_expectations()
    assert e1.shape == (0, 10) and e2.shape == (0, 9)
    eng.close()
