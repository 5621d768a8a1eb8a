"""Writes tests/golden/ed_energies.json: exact ground energies computed by the oracle's
exact diagonalisation (oracle.exact), from the operator-string Hamiltonians in workloads."""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import workloads as wl  # noqa: E402
from oracle import exact  # noqa: E402


def main():
    out = {}
    L = 16
    out["heisenberg_chain_L16_Sz0"] = exact.ground_energy(L, wl.spin_half(), wl.heisenberg_terms(wl.chain_bonds(L)))
    L = 12
    out["heisenberg_chain_L12_Sz0"] = exact.ground_energy(L, wl.spin_half(), wl.heisenberg_terms(wl.chain_bonds(L)))
    out["heisenberg_cylinder_4x3_Sz0"] = exact.ground_energy(12, wl.spin_half(), wl.heisenberg_terms(wl.square_cylinder_bonds(4, 3)))
    out["heisenberg_triangular_4x3_Sz0"] = exact.ground_energy(12, wl.spin_half(), wl.heisenberg_terms(wl.triangular_cylinder_bonds(4, 3)))
    out["spin1_heisenberg_chain_L10_Sz0"] = exact.ground_energy(10, wl.spin_one(), wl.heisenberg_terms(wl.chain_bonds(10)))
    with open(os.path.join(HERE, "ed_energies.json"), "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)
        f.write("\n")


if __name__ == "__main__":
    main()
