"""Independent references for the oracle -- test infrastructure.

* Exact diagonalisation of H = sum of operator strings, built with sparse Kronecker products
  (never through the MPO), restricted to one total-charge sector.
* Transverse-field Ising open chain H = -J sum Z_i Z_{i+1} - h sum X_i: Jordan-Wigner maps it
  to free Majorana fermions, E_0 = -sum_k sigma_k(M) with M the L x L upper-bidiagonal matrix
  (diagonal h, superdiagonal J).
* AKLT open chain H = sum [S.S + (S.S)^2/3] = sum (2 P_2 - 2/3): E_0 = -2(L-1)/3 exactly.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def sector_states(L, qn, qtot):
    """Indices (site 0 most significant) of the product states with total charge qtot."""
    d = len(qn)
    q = np.zeros(1, dtype=np.int64)
    for _ in range(L):
        q = (q[:, None] + np.asarray(qn)[None, :]).ravel()
    return np.nonzero(q == qtot)[0]


def hamiltonian_sparse(L, site, terms):
    d = site.d
    H = sp.csr_matrix((d ** L, d ** L))
    ident = sp.identity(d, format="csr")
    for coef, ops in terms:
        by_site = dict(ops)
        mat = None
        for i in range(L):
            o = sp.csr_matrix(site.op(by_site[i])) if i in by_site else ident
            mat = o if mat is None else sp.kron(mat, o, format="csr")
        H = H + coef * mat
    return H.tocsr()


def ground_energy(L, site, terms, qtot=0, k=1):
    """Lowest eigenvalue(s) of H in the sector of total charge qtot."""
    H = hamiltonian_sparse(L, site, terms)
    idx = sector_states(L, site.qn, qtot)
    Hs = H[idx][:, idx]
    n = Hs.shape[0]
    if n <= 2000:
        ev = np.linalg.eigvalsh(Hs.toarray())
        return ev[:k] if k > 1 else float(ev[0])
    ev = spla.eigsh(Hs, k=k, which="SA", tol=1e-13, maxiter=100000, return_eigenvectors=False)
    ev = np.sort(ev)
    return ev if k > 1 else float(ev[0])


def tfim_energy(L, J, h):
    M = np.diag(np.full(L, float(h))) + np.diag(np.full(L - 1, float(J)), 1)
    return -float(np.sum(np.linalg.svd(M, compute_uv=False)))


def aklt_energy(L):
    return -2.0 * (L - 1) / 3.0
