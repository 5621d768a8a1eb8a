"""Gradients of the projected-Hamiltonian application -- test infrastructure.

For y = H_eff(L, W1, W2, R) x (the Sec. II matvec, `dmrg.heff_apply`) and a scalar
Phi = <ybar, y>, Phi is linear in each of x, L, R, W1 and W2.  Every term of the definition,
c1 c2 L_w X R_w''^T with c1 = W1[w,s1,s1',w1], c2 = W2[w1,s2,s2',w2] and X the x block, gives
  dPhi/dL_w   += c1 c2 Ybar R_w'' X^T        dPhi/dR_w'' += c1 c2 Ybar^T L_w X
  dPhi/dX     += c1 c2 L_w^T Ybar R_w''      dPhi/dW1    += c2 <Ybar, L_w X R_w''^T>,
  dPhi/dW2    += c1 <Ybar, L_w X R_w''^T>,
with Ybar the ybar block of the term's output.  Terms with c1 = 0 or c2 = 0 are absent from the
definition, so zero MPO entries get no gradient (the MPO's sparsity pattern is fixed).
Pinned by central finite differences of `dmrg.heff_apply` along random directions.
"""
from __future__ import annotations

import numpy as np


def heff_backward(Lenv, W1, f0, W2, f2, Renv, psi, ybar, qn):
    """Returns (xbar, Lbar, Rbar, W1bar, W2bar) in the layouts of psi, Lenv, Renv, W1, W2."""
    D0, d, _, D1 = W1.shape
    D2 = W2.shape[3]
    xbar = {k: np.zeros_like(v) for k, v in psi.items()}
    Lbar = {k: np.zeros_like(v) for k, v in Lenv.items()}
    Rbar = {k: np.zeros_like(v) for k, v in Renv.items()}
    W1bar = np.zeros_like(W1)
    W2bar = np.zeros_like(W2)
    for (qa, s1p, s2p), X in psi.items():
        qc = qa + qn[s1p] + qn[s2p]
        for w in range(D0):
            qab = qa + int(f0[w])
            Lb = Lenv.get((qab, w))
            if Lb is None:
                continue
            for s1 in range(d):
                for w1 in range(D1):
                    c1 = W1[w, s1, s1p, w1]
                    if c1 == 0.0:
                        continue
                    for s2 in range(d):
                        Yb = ybar.get((qab, s1, s2))
                        if Yb is None:
                            continue
                        for w2 in range(D2):
                            c2 = W2[w1, s2, s2p, w2]
                            if c2 == 0.0:
                                continue
                            Rb = Renv.get((qc + int(f2[w2]), w2))
                            if Rb is None:
                                continue
                            c = c1 * c2
                            Lbar[(qab, w)] += c * (Yb @ Rb @ X.T)
                            Rbar[(qc + int(f2[w2]), w2)] += c * (Yb.T @ Lb @ X)
                            xbar[(qa, s1p, s2p)] += c * (Lb.T @ Yb @ Rb)
                            v = float(np.sum(Yb * (Lb @ X @ Rb.T)))
                            W1bar[w, s1, s1p, w1] += c2 * v
                            W2bar[w1, s2, s2p, w2] += c1 * v
    return xbar, Lbar, Rbar, W1bar, W2bar
