"""Serial two-site DMRG in plain FP64 NumPy, U(1) block-sparse -- test infrastructure.

Data structures (charges are 2*S^z integers):
  bond      dict q -> m_q, sectors ascending
  site      dict (q_left, s) -> ndarray [m_q_left, m_q_right], q_right = q_left + qn[s]
  two-site  dict (q_a, s1, s2) -> ndarray [m_q_a, m_q_c],      q_c = q_a + qn[s1] + qn[s2]
  L env     dict (q_bra, w) -> ndarray [m_q_bra, m_q_ket],     q_ket = q_bra - f(w)
  R env     dict (q_bra, w) -> ndarray [m_q_bra, m_q_ket],     q_ket = q_bra - f(w)
The MPO convention is the one of ``workloads``: W[w, s, s', w'] = <s|op|s'> and
q(s) - q(s') = f(w') - f(w).  Everything is real.

Paper references: the wavefunction at a bond, Sec. II Eq. (wf); the projected-Hamiltonian
Lanczos/Davidson step, Sec. II; the SVD Psi = A Lambda B and truncation to the m largest
singular values, Sec. II Eq. (svd); choosing A or B to grow a block and the wavefunction
A Lambda or Lambda B for the next bond, Sec. II; the transformation of projected operators by
A or B, Sec. II (operator transformation paragraph).
"""
from __future__ import annotations

import numpy as np

# Truncation rule constants (fixed readings of the paper's unspecified details)
REL_CUTOFF = 1e-12     # discard lambda / lambda_max below this (keeps V = 1/lambda finite)
DEGEN_TOL = 1e-10      # relative gap under which the value at the cut counts as degenerate


def thin_svd(M):
    """M = U diag(S) Vt (thin), S descending -- the SVD of Eq. (svd) as a library step: LAPACK's
    divide-and-conquer driver, or, where that driver reports non-convergence (it does, rarely, on
    valid input with some LAPACK builds), the QR-iteration driver, which computes the same
    factorisation.  Non-finite input is an error, never retried."""
    if not np.all(np.isfinite(M)):
        raise FloatingPointError("SVD of a matrix with non-finite entries")
    try:
        return np.linalg.svd(M, full_matrices=False)
    except np.linalg.LinAlgError:
        import scipy.linalg
        return scipy.linalg.svd(M, full_matrices=False, lapack_driver="gesvd")


# ----------------------------------------------------------------------------------------
# Projected Hamiltonian (Sec. II): out = sum L[a',w,a] W1[w,s1,s1',w'] W2[w',s2,s2',w''] R[c',w'',c] psi[a,s1',s2',c]
# ----------------------------------------------------------------------------------------


def heff_apply(Lenv, W1, f0, W2, f2, Renv, psi, qn):
    """Apply the two-site projected Hamiltonian to psi, summing the definition over all
    index values whose blocks are allowed by charge conservation."""
    D0, d, _, D1 = W1.shape
    D2 = W2.shape[3]
    out = {}
    for (qa, s1p, s2p), blk in psi.items():
        qc = qa + qn[s1p] + qn[s2p]
        for w in range(D0):
            qab = qa + int(f0[w])
            Lb = Lenv.get((qab, w))
            if Lb is None:
                continue
            X = Lb @ blk                                   # sum over a
            for s1 in range(d):
                for w1 in range(D1):
                    c1 = W1[w, s1, s1p, w1]
                    if c1 == 0.0:
                        continue
                    for s2 in range(d):
                        for w2 in range(D2):
                            c2 = W2[w1, s2, s2p, w2]
                            if c2 == 0.0:
                                continue
                            qcb = qc + int(f2[w2])
                            Rb = Renv.get((qcb, w2))
                            if Rb is None:
                                continue
                            key = (qab, s1, s2)
                            term = (c1 * c2) * (X @ Rb.T)   # sum over c
                            if key in out:
                                out[key] = out[key] + term
                            else:
                                out[key] = term
    # blocks of the output space that received nothing are zero
    for key, blk in psi.items():
        if key not in out:
            out[key] = np.zeros_like(blk)
    return {k: out[k] for k in psi}


def heff_diag(Lenv, W1, f0, W2, f2, Renv, psi, qn):
    """Diagonal of the projected Hamiltonian on the blocks of psi (Davidson preconditioner)."""
    D0, d, _, D1 = W1.shape
    D2 = W2.shape[3]
    out = {}
    for (qa, s1, s2), blk in psi.items():
        qc = qa + qn[s1] + qn[s2]
        acc = np.zeros(blk.shape)
        for w in range(D0):
            if f0[w] != 0 or (qa, w) not in Lenv:
                continue
            ld = np.diag(Lenv[(qa, w)])
            for w1 in range(D1):
                c1 = W1[w, s1, s1, w1]
                if c1 == 0.0:
                    continue
                for w2 in range(D2):
                    c2 = W2[w1, s2, s2, w2]
                    if c2 == 0.0 or f2[w2] != 0 or (qc, w2) not in Renv:
                        continue
                    rd = np.diag(Renv[(qc, w2)])
                    acc += (c1 * c2) * np.outer(ld, rd)
        out[(qa, s1, s2)] = acc
    return out


# ----------------------------------------------------------------------------------------
# Block vectors
# ----------------------------------------------------------------------------------------


def vdot(x, y):
    return float(sum(np.sum(x[k] * y[k]) for k in x))


def vaxpy(a, x, y):
    return {k: y[k] + a * x[k] for k in y}


def vscale(a, x):
    return {k: a * v for k, v in x.items()}


def vflat(x):
    return np.concatenate([v.ravel() for v in x.values()]) if x else np.zeros(0)


def vunflat(flat, like):
    out, off = {}, 0
    for k, v in like.items():
        out[k] = flat[off: off + v.size].reshape(v.shape)
        off += v.size
    return out


# ----------------------------------------------------------------------------------------
# Davidson (the Sec. II local eigensolver on the projected Hamiltonian)
# ----------------------------------------------------------------------------------------


def davidson(matvec, x0, diag, tol=1e-10, max_iter=100, kmax=8, precond_floor=1e-4):
    """Lowest eigenpair of a symmetric operator by Davidson's method.

    Vectors are flat FP64 arrays.  Basis V (orthonormal), images AV; Rayleigh-Ritz on
    G = V^T A V; residual r = A u - theta u; stop when |r| <= tol * max(1, |theta|);
    correction t = r / (theta - diag) with |theta - diag| floored at precond_floor;
    two passes of classical Gram-Schmidt; restart from the Ritz vector when the basis
    holds kmax vectors.  Returns (theta, u, iterations, residual_norm)."""
    x = x0 / np.linalg.norm(x0)
    V = [x]
    AV = [matvec(x)]
    theta, u, rn = None, x, np.inf
    it = 0
    for it in range(1, max_iter + 1):
        k = len(V)
        G = np.empty((k, k))
        for i in range(k):
            for j in range(k):
                G[i, j] = V[i] @ AV[j]
        G = 0.5 * (G + G.T)
        evals, evecs = np.linalg.eigh(G)
        theta = evals[0]
        y = evecs[:, 0]
        u = sum(y[i] * V[i] for i in range(k))
        Au = sum(y[i] * AV[i] for i in range(k))
        r = Au - theta * u
        rn = np.linalg.norm(r)
        if rn <= tol * max(1.0, abs(theta)) or it == max_iter:
            break
        den = theta - diag
        small = np.abs(den) < precond_floor
        den[small] = np.where(den[small] >= 0, precond_floor, -precond_floor)
        t = r / den
        if k >= kmax:
            nu = np.linalg.norm(u)
            V = [u / nu]
            AV = [Au / nu]
        for _ in range(2):
            for v in V:
                t = t - (v @ t) * v
        nt = np.linalg.norm(t)
        if nt < 1e-14:
            break
        V.append(t / nt)
        AV.append(matvec(V[-1]))
    return float(theta), u / np.linalg.norm(u), it, float(rn)


# ----------------------------------------------------------------------------------------
# Two-site SVD and truncation (Sec. II, Eq. svd)
# ----------------------------------------------------------------------------------------


def sector_layout(psi_keys, bl, br, qn):
    """Group the (q_a, s1) rows and (s2, q_c) columns of the two-site matrix
    Psi^{(alpha_2 s_3)(s_4 alpha_4)} by the middle charge q_m = q_a + qn[s1]."""
    sectors = {}
    for (qa, s1, s2) in psi_keys:
        qm = qa + qn[s1]
        sec = sectors.setdefault(qm, {"rows": set(), "cols": set()})
        sec["rows"].add((qa, s1))
        sec["cols"].add((s2, qm + qn[s2]))
    out = {}
    for qm in sorted(sectors):
        rows = sorted(sectors[qm]["rows"])
        cols = sorted(sectors[qm]["cols"])
        roff, o = {}, 0
        for (qa, s1) in rows:
            roff[(qa, s1)] = o
            o += bl[qa]
        nr = o
        coff, o = {}, 0
        for (s2, qc) in cols:
            coff[(s2, qc)] = o
            o += br[qc]
        out[qm] = (roff, nr, coff, o)
    return out


def svd_sectors(psi, bl, br, qn, svd=None):
    """Per middle-charge sector: gather the matrix and take its SVD (full numpy SVD unless
    another routine is passed, e.g. the Appendix's accurate SVD)."""
    layout = sector_layout(list(psi.keys()), bl, br, qn)
    res = {}
    for qm, (roff, nr, coff, nc) in layout.items():
        M = np.zeros((nr, nc))
        for (qa, s1), r0 in roff.items():
            for (s2, qc), c0 in coff.items():
                blk = psi.get((qa, s1, s2))
                if blk is not None:
                    M[r0: r0 + bl[qa], c0: c0 + br[qc]] = blk
        if svd is None:
            U, S, Vt = thin_svd(M)
        else:
            U, S, Vt = svd(M)
        res[qm] = (U, S, Vt, roff, coff)
    return res


def truncate(svals, m_max, rel_cutoff=REL_CUTOFF, degen_tol=DEGEN_TOL):
    """Select the kept singular values over all sectors.

    svals: dict q -> 1D array (descending).  Rule: drop lambda <= rel_cutoff * lambda_max;
    order by (lambda descending, q ascending, index ascending); keep the first m_max; if the
    first discarded value is degenerate with the last kept (relative gap <= degen_tol), drop
    every kept value that is degenerate with it as well.  Returns (dict q -> kept count,
    discarded weight / total weight)."""
    allv = [(float(v), q, i) for q, s in svals.items() for i, v in enumerate(s)]
    total = sum(v * v for v, _, _ in allv)
    if not allv or total == 0.0:
        return {}, 0.0
    lmax = max(v for v, _, _ in allv)
    cand = [t for t in allv if t[0] > rel_cutoff * lmax]
    cand.sort(key=lambda t: (-t[0], t[1], t[2]))
    kept = cand[:m_max]
    if len(cand) > m_max:
        nxt = cand[m_max][0]
        kept = [t for t in kept if t[0] > nxt * (1.0 + degen_tol)]
    counts = {}
    for _, q, _ in kept:
        counts[q] = counts.get(q, 0) + 1
    kw = sum(v * v for v, _, _ in kept)
    return dict(sorted(counts.items())), (total - kw) / total


def split_two_site(psi, bl, br, qn, m_max, svd=None):
    """SVD of the two-site wavefunction with truncation.  Returns (A, lam, B, bond, err):
    A[(q_a, s1)] : [m_qa, k_qm] left singular vectors, lam[q_m] : kept singular values
    normalised to sum(lam^2) = 1, B[(q_m, s2)] : [k_qm, m_qc] right singular vectors."""
    secs = svd_sectors(psi, bl, br, qn, svd)
    counts, err = truncate({q: v[1] for q, v in secs.items()}, m_max)
    A, B, lam = {}, {}, {}
    for qm, k in counts.items():
        U, S, Vt, roff, coff = secs[qm]
        lam[qm] = S[:k].copy()
        for (qa, s1), r0 in roff.items():
            A[(qa, s1)] = U[r0: r0 + bl[qa], :k].copy()
        for (s2, qc), c0 in coff.items():
            B[(qm, s2)] = Vt[:k, c0: c0 + br[qc]].copy()
    nrm = np.sqrt(sum(np.sum(v * v) for v in lam.values()))
    lam = {q: v / nrm for q, v in lam.items()}
    return A, lam, B, dict(counts), err


# ----------------------------------------------------------------------------------------
# Projected-operator updates (Sec. II operator transformation by A or B)
# ----------------------------------------------------------------------------------------


def env_left(Lenv, A, W, fL, fR, qn):
    """L_{j+1}[b', w', b] = sum A[a', s, b'] L_j[a', w, a] W[w, s, s', w'] A[a, s', b]."""
    d = W.shape[1]
    out = {}
    for (qab, w), Lb in Lenv.items():
        qak = qab - int(fL[w])
        for sp in range(d):
            Ak = A.get((qak, sp))
            if Ak is None:
                continue
            T = Lb @ Ak
            for s in range(d):
                Ab = A.get((qab, s))
                if Ab is None:
                    continue
                for wp in range(W.shape[3]):
                    c = W[w, s, sp, wp]
                    if c == 0.0:
                        continue
                    key = (qab + qn[s], wp)
                    term = c * (Ab.T @ T)
                    out[key] = out[key] + term if key in out else term
    return out


def env_right(Renv, B, W, fL, fR, qn):
    """R_j[a', w, a] = sum B[a', s, c'] R_{j+1}[c', w', c] W[w, s, s', w'] B[a, s', c]."""
    d = W.shape[1]
    byright = {}
    for (ql, s), blk in B.items():
        byright.setdefault(ql + qn[s], []).append((ql, s, blk))
    out = {}
    for (qcb, wp), Rb in Renv.items():
        qck = qcb - int(fR[wp])
        for (qak, sp, Bk) in byright.get(qck, []):
            T = Bk @ Rb.T                                  # [m_qak, m_qcb]
            for (qab, s, Bb) in byright.get(qcb, []):
                for w in range(W.shape[0]):
                    c = W[w, s, sp, wp]
                    if c == 0.0:
                        continue
                    key = (qab, w)
                    term = c * (Bb @ T.T)
                    out[key] = out[key] + term if key in out else term
    return out


# ----------------------------------------------------------------------------------------
# Serial DMRG driver
# ----------------------------------------------------------------------------------------


def right_canonicalize(mps_sites, bonds, qn):
    """Bring a block MPS to right-canonical form with the orthogonality centre on site 0 by
    exact (untruncated) SVDs from the right.  Returns (sites, bonds) as new objects."""
    sites = [dict(s) for s in mps_sites]
    bonds = [dict(b) for b in bonds]
    L = len(sites)
    for j in range(L - 1, 0, -1):
        bl, br = bonds[j], bonds[j + 1]
        newdims = {}
        newblk = {}
        carry = {}
        for ql, ml in bl.items():
            cols = [(s, ql + qs) for s, qs in enumerate(qn) if (ql + qs) in br and (ql, s) in sites[j]]
            if not cols:
                continue
            M = np.concatenate([sites[j][(ql, s)] for s, _ in cols], axis=1)
            U, S, Vt = thin_svd(M)
            k = len(S)
            newdims[ql] = k
            c0 = 0
            for s, qr in cols:
                newblk[(ql, s)] = Vt[:, c0: c0 + br[qr]].copy()
                c0 += br[qr]
            carry[ql] = (U, S)
        # the overall scale is irrelevant (the state is normalised at the end); dividing each
        # carry by the norm of its singular values keeps long random chains from overflowing
        nrm_j = np.sqrt(sum(float(np.sum(S * S)) for _, S in carry.values()))
        carry = {q: U * (S / nrm_j) for q, (U, S) in carry.items()}
        sites[j] = newblk
        bonds[j] = newdims
        prev = {}
        for (qx, s), blk in sites[j - 1].items():
            qr = qx + qn[s]
            if qr in carry:
                prev[(qx, s)] = blk @ carry[qr]
        sites[j - 1] = prev
    nrm = np.sqrt(sum(np.sum(b * b) for b in sites[0].values()))
    sites[0] = {k: v / nrm for k, v in sites[0].items()}
    return sites, bonds


def two_site(left, right, qn):
    """Psi[(q_a, s1, s2)] = sum over the middle bond of left[(q_a, s1)] right[(q_m, s2)]."""
    out = {}
    for (qa, s1), X in left.items():
        qm = qa + qn[s1]
        for s2 in range(len(qn)):
            Y = right.get((qm, s2))
            if Y is not None:
                out[(qa, s1, s2)] = X @ Y
    return out


class SerialDMRG:
    """Finite-size two-site DMRG (Sec. II) on one MPS, orthogonality centre tracked."""

    def __init__(self, mpo, mps, kmax=8):
        self.mpo = mpo
        self.qn = list(mpo.site.qn)
        self.L = mpo.L
        self.kmax = kmax
        self.sites, self.bonds = right_canonicalize(mps.sites, mps.bonds, self.qn)
        L = self.L
        self.Lenv = [None] * (L + 1)
        self.Renv = [None] * (L + 1)
        self.Lenv[0] = {(0, 0): np.ones((1, 1))}
        qt = list(self.bonds[L].keys())[0]
        self.Renv[L] = {(qt, 0): np.ones((1, 1))}
        for j in range(L - 1, 0, -1):
            self.Renv[j] = env_right(self.Renv[j + 1], self.sites[j], mpo.W[j],
                                     mpo.flux[j], mpo.flux[j + 1], self.qn)
        self.oc = 0
        self.lam = [None] * (L + 1)
        self.history = []

    # local problem at bond (j, j+1)
    def local_ops(self, j):
        m = self.mpo
        return (self.Lenv[j], m.W[j], m.flux[j], m.W[j + 1], m.flux[j + 2], self.Renv[j + 2])

    def energy_of(self, j, psi):
        Lb, W1, f0, W2, f2, Rb = self.local_ops(j)
        Hp = heff_apply(Lb, W1, f0, W2, f2, Rb, psi, self.qn)
        return vdot(psi, Hp) / vdot(psi, psi)

    def solve_local(self, j, psi, tol, max_iter):
        Lb, W1, f0, W2, f2, Rb = self.local_ops(j)
        qn = self.qn

        def mv(x):
            return vflat(heff_apply(Lb, W1, f0, W2, f2, Rb, vunflat(x, psi), qn))

        dg = vflat(heff_diag(Lb, W1, f0, W2, f2, Rb, psi, qn))
        theta, u, it, rn = davidson(mv, vflat(psi), dg, tol=tol, max_iter=max_iter, kmax=self.kmax)
        return theta, vunflat(u, psi), it, rn

    def bond_step(self, j, direction, m_max, tol=1e-10, max_iter=100, svd=None):
        qn = self.qn
        psi = two_site(self.sites[j], self.sites[j + 1], qn)
        theta, psi, it, rn = self.solve_local(j, psi, tol, max_iter)
        A, lam, B, counts, err = split_two_site(psi, self.bonds[j], self.bonds[j + 2], qn, m_max, svd)
        self.bonds[j + 1] = counts
        self.lam[j + 1] = lam
        m = self.mpo
        if direction == "right":
            self.sites[j] = A
            self.sites[j + 1] = {(qm, s2): lam[qm][:, None] * blk for (qm, s2), blk in B.items()}
            self.Lenv[j + 1] = env_left(self.Lenv[j], A, m.W[j], m.flux[j], m.flux[j + 1], qn)
            self.oc = j + 1
        else:
            self.sites[j + 1] = B
            self.sites[j] = {(qa, s1): blk * lam[qa + qn[s1]][None, :] for (qa, s1), blk in A.items()}
            self.Renv[j + 1] = env_right(self.Renv[j + 2], B, m.W[j + 1], m.flux[j + 1], m.flux[j + 2], qn)
            self.oc = j
        rec = dict(bond=j, dir=direction, energy=theta, iters=it, resid=rn, trunc=err,
                   m=sum(counts.values()))
        self.history.append(rec)
        return rec

    def sweep(self, m_max, tol=1e-10, max_iter=100, svd=None):
        """One full sweep: bonds 0..L-2 moving right, then L-2..0 moving left."""
        recs = []
        for j in range(self.L - 1):
            recs.append(self.bond_step(j, "right", m_max, tol, max_iter, svd))
        for j in range(self.L - 2, -1, -1):
            recs.append(self.bond_step(j, "left", m_max, tol, max_iter, svd))
        return dict(energy=recs[-1]["energy"], max_trunc=max(r["trunc"] for r in recs),
                    m=max(r["m"] for r in recs), steps=recs)

    def expectation_energy(self):
        """<Psi|H|Psi> with the orthogonality centre on site oc (requires oc <= L-2)."""
        j = min(self.oc, self.L - 2)
        if self.oc == j:
            psi = two_site(self.sites[j], self.sites[j + 1], self.qn)
        else:
            psi = two_site(self.sites[j], self.sites[j + 1], self.qn)
        return self.energy_of(j, psi)
