"""Input generators: lattices, MPO encoding (checked against direct Kronecker sums)."""
import numpy as np
import pytest

import workloads as wl
from oracle import exact
from tests import _helpers as H


def test_square_cylinder_bond_count_and_coordination():
    Lx, Ly = 24, 8
    bonds = wl.square_cylinder_bonds(Lx, Ly)
    assert len(bonds) == (Lx - 1) * Ly + Lx * Ly          # horizontal + periodic vertical
    deg = np.zeros(Lx * Ly, int)
    for i, j in bonds:
        deg[i] += 1
        deg[j] += 1
    assert deg.max() == 4 and deg.min() == 3              # bulk 4, open edges 3


def test_triangular_cylinder_coordination():
    Lx, Ly = 12, 6
    bonds = wl.triangular_cylinder_bonds(Lx, Ly)
    assert len(bonds) == (Lx - 1) * Ly * 2 + Lx * Ly
    deg = np.zeros(Lx * Ly, int)
    for i, j in bonds:
        deg[i] += 1
        deg[j] += 1
    assert deg.max() == 6


def test_snake_order_is_a_permutation():
    Lx, Ly = 5, 4
    idx = sorted(wl.snake_index(x, y, Ly) for x in range(Lx) for y in range(Ly))
    assert idx == list(range(Lx * Ly))


@pytest.mark.parametrize("name", ["heis", "tfim", "aklt", "cyl", "tri", "jq2", "field"])
def test_mpo_equals_operator_sum(name):
    """The FSM MPO contracted to a matrix equals the Kronecker-product Hamiltonian."""
    if name == "heis":
        L = 6; site = wl.spin_half(); terms = wl.heisenberg_terms(wl.chain_bonds(L))
    elif name == "tfim":
        L = 6; site = wl.spin_half_pauli(); terms = wl.tfim_terms(L, 0.8, 1.3)
    elif name == "aklt":
        L = 4; site = wl.spin_one(); terms = wl.aklt_terms(L)
    elif name == "cyl":
        L = 8; site = wl.spin_half(); terms = wl.heisenberg_terms(wl.square_cylinder_bonds(2, 4))
    elif name == "tri":
        L = 9; site = wl.spin_half(); terms = wl.heisenberg_terms(wl.triangular_cylinder_bonds(3, 3))
    elif name == "field":
        L = 8; site = wl.spin_half()
        terms = (wl.heisenberg_terms(wl.square_cylinder_bonds(2, 4))
                 + wl.field_terms(np.random.default_rng(4).uniform(-0.5, 0.5, L)))
    else:
        L = 8
        site = wl.spin_half()
        rng = np.random.default_rng(3)
        nb = len(wl.square_cylinder_bonds(2, 4))
        npair = 2 * len(wl.square_plaquettes(2, 4))
        terms, _ = wl.jq2_terms(2, 4, rng.uniform(0.5, 2, nb), rng.uniform(0.5, 2, npair))
    mpo = wl.build_mpo(L, site, terms)
    Hm = H.mpo_to_matrix(mpo)
    Hs = exact.hamiltonian_sparse(L, site, terms).toarray()
    assert np.abs(Hm - Hs).max() < 1e-12


def test_mpo_selection_rule():
    mpo = wl.heisenberg_square_cylinder(4, 4)
    qn = mpo.site.qn
    for j, W in enumerate(mpo.W):
        nz = np.argwhere(W != 0)
        for w, s, sp, wp in nz:
            assert qn[s] - qn[sp] == mpo.flux[j + 1][wp] - mpo.flux[j][w]


def test_cylinder_24x8_mpo_bond_dimension():
    mpo = wl.heisenberg_square_cylinder(24, 8)
    assert mpo.L == 192
    assert max(mpo.D) <= 2 + 3 * 9


def test_random_mps_blocks_respect_charges():
    mps = wl.random_mps(12, (1, -1), 0, 20, seed=0)
    for j, blocks in enumerate(mps.sites):
        for (ql, s), blk in blocks.items():
            qr = ql + (1, -1)[s]
            assert blk.shape == (mps.bonds[j][ql], mps.bonds[j + 1][qr])
    assert mps.bonds[0] == {0: 1} and mps.bonds[12] == {0: 1}


def test_random_mps_is_seeded():
    a = wl.random_mps(10, (1, -1), 0, 16, seed=5)
    b = wl.random_mps(10, (1, -1), 0, 16, seed=5)
    for x, y in zip(a.sites, b.sites):
        for k in x:
            assert np.array_equal(x[k], y[k])
