"""Real-space parallel DMRG, regions executed one after another -- test infrastructure.

Follows Sec. II of the paper:
* at a region boundary (a bond) the two-site SVD Psi = A Lambda B is rewritten with the
  identity Lambda V = 1, V = Lambda^{-1} (Eqs. inverse and isvd): the left region keeps
  psi_3 = A Lambda, the right region psi_4 = Lambda B, and V is stored on the bond;
* each region sweeps independently; its projected operators at the boundary stay those of
  the neighbour at split time;
* when two regions meet, the merged wavefunction is Psi' = psi'_3 V psi'_4 with the original
  V (Eq. merge), the left environment comes from the left region and the right one from the
  right region, Psi' is optimised by Davidson on the shared bond, and split again (Fig. 2);
* Fig. 4's staggered pattern: odd regions (1-based) start at the left end of their block,
  even ones at the right end; all sweep to their other end, meet and merge, sweep back and
  merge with their other neighbour.  A region waits for its neighbour before merging.
* shared bonds use the Appendix's accurate SVD.

Readings where the paper leaves details open:
* boundaries are bonds b_k = round(k L / R); region k holds sites [b_k, b_{k+1});
* set-up: serial warm-up sweeps; the last warm-up left half-sweep performs the Lambda V
  Lambda split at every boundary it crosses (without warm-up, that pass moves the gauge by
  untruncated SVDs and no Davidson), so every region starts with its centre at its left end;
  even regions (1-based) then sweep once to their right end to take the staggered positions;
* one parallel sweep = Fig. 4 (a)-(d); its energy is the Davidson energy of its last merge;
* merge fidelity = 1 - |<Psi'|Psi>| with both normalised (Fig. 3).
"""
from __future__ import annotations

import numpy as np

from . import dmrg as D
from .accsvd import accurate_svd


class Region:
    def __init__(self, p, q):
        self.p, self.q = p, q          # sites p..q inclusive
        self.sites = {}
        self.bonds = {}                # global bond index -> sector dims, bonds p..q+1
        self.Lenv = {}
        self.Renv = {}
        self.oc = p


class ParallelDMRG:
    def __init__(self, mpo, mps, n_regions, kmax=8):
        self.serial = D.SerialDMRG(mpo, mps, kmax=kmax)
        self.mpo = mpo
        self.qn = list(mpo.site.qn)
        self.L = mpo.L
        self.R = n_regions
        self.kmax = kmax
        self.bounds = [int(round(k * self.L / n_regions)) for k in range(n_regions + 1)]
        for k in range(n_regions):
            if self.bounds[k + 1] - self.bounds[k] < 2:
                raise ValueError("every region needs at least two sites")
        self.regions = None
        self.V = {}
        self.merges = []

    # ------------------------------------------------------------------ helpers
    def _gauge_step(self, eng, j, direction, m_max):
        """Move the orthogonality centre across bond j by an SVD of the current two-site
        wavefunction (no Davidson)."""
        qn = self.qn
        psi = D.two_site(eng.sites[j], eng.sites[j + 1], qn)
        A, lam, B, counts, err = D.split_two_site(psi, eng.bonds[j], eng.bonds[j + 2], qn, m_max)
        eng.bonds[j + 1] = counts
        m = self.mpo
        if direction == "right":
            eng.sites[j] = A
            eng.sites[j + 1] = {(qm, s2): lam[qm][:, None] * b for (qm, s2), b in B.items()}
            eng.Lenv[j + 1] = D.env_left(eng.Lenv[j], A, m.W[j], m.flux[j], m.flux[j + 1], qn)
            eng.oc = j + 1
        else:
            eng.sites[j + 1] = B
            eng.sites[j] = {(qa, s1): b * lam[qa + qn[s1]][None, :] for (qa, s1), b in A.items()}
            eng.Renv[j + 1] = D.env_right(eng.Renv[j + 2], B, m.W[j + 1], m.flux[j + 1], m.flux[j + 2], qn)
            eng.oc = j
        return A, lam, B

    def setup(self, m_max, warmup_sweeps=0, tol=1e-10, max_iter=100):
        eng = self.serial
        L = self.L
        for _ in range(max(0, warmup_sweeps - 1)):
            eng.sweep(m_max, tol, max_iter)
        for j in range(L - 1):
            if warmup_sweeps > 0:
                eng.bond_step(j, "right", m_max, tol, max_iter)
            else:
                self._gauge_step(eng, j, "right", 10 ** 9)
        regions = [Region(self.bounds[k], self.bounds[k + 1] - 1) for k in range(self.R)]
        m = self.mpo
        qn = self.qn
        bset = set(self.bounds[1:-1])
        for j in range(L - 2, -1, -1):
            b = j + 1
            if warmup_sweeps > 0:
                psi = D.two_site(eng.sites[j], eng.sites[j + 1], qn)
                svd = accurate_svd if b in bset else None
                theta, psi, it, rn = eng.solve_local(j, psi, tol, max_iter)
                A, lam, B, counts, err = D.split_two_site(psi, eng.bonds[j], eng.bonds[j + 2], qn, m_max, svd)
                eng.bonds[j + 1] = counts
                eng.sites[j + 1] = B
                eng.sites[j] = {(qa, s1): x * lam[qa + qn[s1]][None, :] for (qa, s1), x in A.items()}
                eng.Renv[j + 1] = D.env_right(eng.Renv[j + 2], B, m.W[j + 1], m.flux[j + 1], m.flux[j + 2], qn)
                eng.oc = j
            else:
                A, lam, B = self._gauge_step(eng, j, "left", 10 ** 9)
            if b in bset:
                k = self.bounds.index(b)
                reg = regions[k]
                self.V[b] = {q: 1.0 / v for q, v in lam.items()}
                reg.Lenv[b] = D.env_left(eng.Lenv[j], A, m.W[j], m.flux[j], m.flux[j + 1], qn)
                reg.sites[b] = {(qm, s2): lam[qm][:, None] * x for (qm, s2), x in B.items()}
        # copy the remaining tensors / environments into their regions
        for k, reg in enumerate(regions):
            for s in range(reg.p, reg.q + 1):
                if s not in reg.sites:
                    reg.sites[s] = dict(eng.sites[s])
            for b in range(reg.p, reg.q + 2):
                reg.bonds[b] = dict(eng.bonds[b])
            if k == 0:
                reg.Lenv[0] = eng.Lenv[0]
            for b in range(reg.p + 1, reg.q + 2):
                reg.Renv[b] = eng.Renv[b]
            reg.oc = reg.p
        self.regions = regions
        # staggered start: even regions (1-based) go to their right end
        for k in range(1, self.R, 2):
            self.half_sweep(k, "right", m_max, tol, max_iter)

    # ------------------------------------------------------------------ region sweeps
    def _local(self, reg, j):
        m = self.mpo
        return (reg.Lenv[j], m.W[j], m.flux[j], m.W[j + 1], m.flux[j + 2], reg.Renv[j + 2])

    def region_step(self, reg, j, direction, m_max, tol, max_iter):
        qn = self.qn
        m = self.mpo
        psi = D.two_site(reg.sites[j], reg.sites[j + 1], qn)
        Lb, W1, f0, W2, f2, Rb = self._local(reg, j)

        def mv(x):
            return D.vflat(D.heff_apply(Lb, W1, f0, W2, f2, Rb, D.vunflat(x, psi), qn))

        dg = D.vflat(D.heff_diag(Lb, W1, f0, W2, f2, Rb, psi, qn))
        theta, u, it, rn = D.davidson(mv, D.vflat(psi), dg, tol=tol, max_iter=max_iter, kmax=self.kmax)
        psi = D.vunflat(u, psi)
        A, lam, B, counts, err = D.split_two_site(psi, reg.bonds[j], reg.bonds[j + 2], qn, m_max)
        reg.bonds[j + 1] = counts
        if direction == "right":
            reg.sites[j] = A
            reg.sites[j + 1] = {(qm, s2): lam[qm][:, None] * b for (qm, s2), b in B.items()}
            reg.Lenv[j + 1] = D.env_left(reg.Lenv[j], A, m.W[j], m.flux[j], m.flux[j + 1], qn)
            reg.oc = j + 1
        else:
            reg.sites[j + 1] = B
            reg.sites[j] = {(qa, s1): b * lam[qa + qn[s1]][None, :] for (qa, s1), b in A.items()}
            reg.Renv[j + 1] = D.env_right(reg.Renv[j + 2], B, m.W[j + 1], m.flux[j + 1], m.flux[j + 2], qn)
            reg.oc = j
        return dict(bond=j, energy=theta, iters=it, trunc=err, m=sum(counts.values()))

    def half_sweep(self, k, direction, m_max, tol=1e-10, max_iter=100):
        reg = self.regions[k]
        recs = []
        if direction == "right":
            assert reg.oc == reg.p
            for j in range(reg.p, reg.q):
                recs.append(self.region_step(reg, j, "right", m_max, tol, max_iter))
        else:
            assert reg.oc == reg.q
            for j in range(reg.q - 1, reg.p - 1, -1):
                recs.append(self.region_step(reg, j, "left", m_max, tol, max_iter))
        return recs

    # ------------------------------------------------------------------ merge (Eq. merge)
    def merge(self, k, m_max, tol=1e-10, max_iter=100):
        """Merge regions k-1 and k at boundary b = bounds[k]; both must have their centre at
        the shared bond."""
        left, right = self.regions[k - 1], self.regions[k]
        b = self.bounds[k]
        assert left.oc == b - 1 and right.oc == b
        qn = self.qn
        m = self.mpo
        V = self.V[b]
        psi3 = left.sites[b - 1]
        psi4 = right.sites[b]
        merged = {}
        for (qa, s1), X in psi3.items():
            qm = qa + qn[s1]
            if qm not in V:
                continue
            for s2 in range(len(qn)):
                Y = psi4.get((qm, s2))
                if Y is not None:
                    merged[(qa, s1, s2)] = (X * V[qm][None, :]) @ Y
        nrm = np.sqrt(D.vdot(merged, merged))
        merged = D.vscale(1.0 / nrm, merged)
        Lb = left.Lenv[b - 1]
        Rb = right.Renv[b + 1]
        W1, f0, W2, f2 = m.W[b - 1], m.flux[b - 1], m.W[b], m.flux[b + 1]

        def mv(x):
            return D.vflat(D.heff_apply(Lb, W1, f0, W2, f2, Rb, D.vunflat(x, merged), qn))

        dg = D.vflat(D.heff_diag(Lb, W1, f0, W2, f2, Rb, merged, qn))
        theta, u, it, rn = D.davidson(mv, D.vflat(merged), dg, tol=tol, max_iter=max_iter, kmax=self.kmax)
        fidelity = 1.0 - abs(float(D.vflat(merged) @ u))
        psi = D.vunflat(u, merged)
        bl = left.bonds[b - 1]
        br = right.bonds[b + 1]
        A, lam, B, counts, err = D.split_two_site(psi, bl, br, qn, m_max, accurate_svd)
        self.V[b] = {q: 1.0 / v for q, v in lam.items()}
        left.bonds[b] = dict(counts)
        right.bonds[b] = dict(counts)
        left.sites[b - 1] = {(qa, s1): x * lam[qa + qn[s1]][None, :] for (qa, s1), x in A.items()}
        right.sites[b] = {(qm, s2): lam[qm][:, None] * x for (qm, s2), x in B.items()}
        left.Renv[b] = D.env_right(right.Renv[b + 1], B, m.W[b], m.flux[b], m.flux[b + 1], qn)
        right.Lenv[b] = D.env_left(left.Lenv[b - 1], A, m.W[b - 1], m.flux[b - 1], m.flux[b], qn)
        rec = dict(boundary=b, energy=theta, fidelity=fidelity, iters=it, trunc=err,
                   m=sum(counts.values()))
        self.merges.append(rec)
        return rec

    # ------------------------------------------------------------------ Fig. 4 sweep
    def sweep(self, m_max, tol=1e-10, max_iter=100):
        R = self.R
        recs = []
        for k in range(R):                                  # (a)
            self.half_sweep(k, "right" if k % 2 == 0 else "left", m_max, tol, max_iter)
        for k in range(1, R, 2):                            # (b) boundaries 1|2, 3|4, ...
            recs.append(self.merge(k, m_max, tol, max_iter))
        for k in range(R):                                  # (c)
            self.half_sweep(k, "left" if k % 2 == 0 else "right", m_max, tol, max_iter)
        for k in range(2, R, 2):                            # (d) boundaries 2|3, 4|5, ...
            recs.append(self.merge(k, m_max, tol, max_iter))
        return dict(energy=recs[-1]["energy"] if recs else None, merges=recs)
