"""Inverse canonical MPS gauge and local expectation values (Sec. IV) -- test infrastructure.

The gauge (Sec. IV, Figs. 8 and 9): every site tensor psi_j is an orthogonality centre (OC) and
every inner bond b carries the diagonal V_b = Lambda_b^-1 of inverse Schmidt weights, so that the
state is psi_0 V_1 psi_1 V_2 ... V_{L-1} psi_{L-1}, with psi_j = Lambda_j Gamma_j Lambda_{j+1}
in the Gamma-Lambda (canonical) notation.  Bond b sits between sites b-1 and b; bonds 0 and L
are trivial (Lambda = 1).

Construction, as Sec. IV builds it: start from the MPS with its OC on the first site (all other
sites right-orthonormal), then at every bond in turn, left to right, contract the two site
tensors, take the SVD Theta = U Lambda W^T (untruncated apart from the REL_CUTOFF reading that
keeps V finite), and multiply one copy of Lambda into each neighbour -- psi_j <- U Lambda,
psi_{j+1} <- Lambda W^T -- with V = Lambda^-1 left on the bond.

Local expectation values (Sec. IV): since every psi_j is an OC, an operator on site j needs only
psi_j, and an operator on sites (j, j+1) only Theta_j = psi_j V_{j+1} psi_{j+1}; all other
tensors represent orthonormal states and drop out.

Pinned in tests/test_oracle_icmps.py against dense state vectors: the gauge leaves the state
unchanged, V_b^-1 are the Schmidt values of the dense state at cut b (numpy SVD of the
reshaped vector), every psi_j is an OC (dense left/right parts orthonormal), one- and two-site
expectation values equal <v|O|v> of the dense state, sum_j <S^z_j> equals the sector's total
S^z, and the bond energies of a converged Heisenberg chain add up to the exact-diagonalisation
energy.
"""
from __future__ import annotations

import numpy as np

from . import dmrg as O


def inverse_canonical(sites, bonds, qn):
    """Returns (psi, V, bonds): psi[j] site dicts (q_left, s) -> block, V[b] dict q -> 1D array
    of inverse Schmidt weights for the inner bonds b = 1..L-1 (V[0] = V[L] = None), and the new
    bond sector dims.  The input MPS may be in any gauge; it is normalised."""
    psi, bonds = O.right_canonicalize(sites, bonds, qn)     # OC on site 0, sites 1.. right-orthonormal
    psi = [dict(s) for s in psi]
    bonds = [dict(b) for b in bonds]
    L = len(psi)
    V = [None] * (L + 1)
    for j in range(L - 1):
        theta = O.two_site(psi[j], psi[j + 1], qn)
        A, lam, B, mid, _ = O.split_two_site(theta, bonds[j], bonds[j + 2], qn, m_max=1 << 60)
        # one copy of Lambda into each neighbour, V = Lambda^-1 on the bond (Fig. 8)
        psi[j] = {(qa, s): blk * lam[qa + qn[s]][None, :] for (qa, s), blk in A.items()}
        psi[j + 1] = {(qm, s): lam[qm][:, None] * blk for (qm, s), blk in B.items()}
        V[j + 1] = {q: 1.0 / v for q, v in lam.items()}
        bonds[j + 1] = dict(mid)
    return psi, V, bonds


def local_expectation(psi_j, op, qn):
    """<O_j> = sum psi_j[a, s, b] O[s, s'] psi_j[a, s', b] / |psi_j|^2 (psi_j an OC).  Blocks
    (q_a, s) and (q_a, s') overlap only where both exist; they then share the right sector when
    qn[s] == qn[s'], the only case with a nonzero contribution."""
    num, den = 0.0, 0.0
    for (qa, s), X in psi_j.items():
        den += float(np.sum(X * X))
        for sp in range(len(qn)):
            if op[s, sp] == 0.0 or qn[s] != qn[sp]:
                continue
            Y = psi_j.get((qa, sp))
            if Y is not None:
                num += op[s, sp] * float(np.sum(X * Y))
    return num / den


def bond_wavefunction(psi_j, V_b, psi_k, qn):
    """Theta = psi_j V_b psi_{j+1} as a two-site dict (q_a, s1, s2) -> block."""
    scaled = {(qa, s): blk * V_b[qa + qn[s]][None, :] for (qa, s), blk in psi_j.items()}
    return O.two_site(scaled, psi_k, qn)


def bond_expectation(theta, op2, qn):
    """<O_{j,j+1}> = sum Theta[a,s1,s2,c] O2[(s1 s2), (s1' s2')] Theta[a,s1',s2',c] / |Theta|^2,
    op2 a [d*d, d*d] matrix with row index s1*d + s2."""
    d = len(qn)
    num, den = 0.0, 0.0
    for (qa, s1, s2), X in theta.items():
        den += float(np.sum(X * X))
        for s1p in range(d):
            for s2p in range(d):
                c = op2[s1 * d + s2, s1p * d + s2p]
                if c == 0.0 or qn[s1] + qn[s2] != qn[s1p] + qn[s2p]:
                    continue
                Y = theta.get((qa, s1p, s2p))
                if Y is not None:
                    num += c * float(np.sum(X * Y))
    return num / den


def all_expectations(psi, V, qn, ops1=(), ops2=()):
    """[len(ops1), L] one-site values and [len(ops2), L-1] nearest-neighbour values."""
    L = len(psi)
    e1 = np.array([[local_expectation(psi[j], o, qn) for j in range(L)] for o in ops1]).reshape(len(ops1), L)
    thetas = [bond_wavefunction(psi[j], V[j + 1], psi[j + 1], qn) for j in range(L - 1)]
    e2 = np.array([[bond_expectation(t, o, qn) for t in thetas] for o in ops2]).reshape(len(ops2), L - 1)
    return e1, e2
