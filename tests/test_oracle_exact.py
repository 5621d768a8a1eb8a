"""Pins for the independent references themselves (ED, closed forms)."""
import numpy as np
import pytest

import workloads as wl
from oracle import exact


def test_two_site_singlet():
    e = exact.ground_energy(2, wl.spin_half(), wl.heisenberg_terms([(0, 1)]))
    assert abs(e - (-0.75)) < 1e-14


@pytest.mark.parametrize("L", [1, 2, 3, 5, 8])
@pytest.mark.parametrize("h", [0.0, 0.5, 1.0, 1.7])
def test_tfim_closed_form_matches_ed(L, h):
    J = 1.0
    terms = wl.tfim_terms(L, J, h)
    e_ed = exact.ground_energy(L, wl.spin_half_pauli(), terms)
    assert abs(exact.tfim_energy(L, J, h) - e_ed) < 1e-11


def test_tfim_special_cases():
    assert abs(exact.tfim_energy(1, 1.0, 0.6) + 0.6) < 1e-15          # single spin: -h
    assert abs(exact.tfim_energy(7, 1.3, 0.0) + 1.3 * 6) < 1e-13        # classical: -J(L-1)


@pytest.mark.parametrize("L", [2, 3, 4, 5, 6])
def test_aklt_energy_matches_ed(L):
    e_ed = exact.ground_energy(L, wl.spin_one(), wl.aklt_terms(L))
    assert abs(e_ed - exact.aklt_energy(L)) < 1e-11


def test_heisenberg_ring_of_four_closed_form():
    # 4-site periodic Heisenberg ring: E0 = -2 J (textbook, total singlet of S=2 ... )
    bonds = [(0, 1), (1, 2), (2, 3), (0, 3)]
    e = exact.ground_energy(4, wl.spin_half(), wl.heisenberg_terms(bonds))
    assert abs(e + 2.0) < 1e-13


def test_sector_restriction():
    L = 6
    terms = wl.heisenberg_terms(wl.chain_bonds(L))
    full = np.linalg.eigvalsh(exact.hamiltonian_sparse(L, wl.spin_half(), terms).toarray())[0]
    assert abs(exact.ground_energy(L, wl.spin_half(), terms, qtot=0) - full) < 1e-12
