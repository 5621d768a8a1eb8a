"""Dense test helpers: expand block tensors to full vectors/matrices for small systems."""
import numpy as np


def _offsets(bond):
    off, o = {}, 0
    for q, m in bond.items():
        off[q] = o
        o += m
    return off, o


def dense_site(blocks, bl, br, qn):
    ol, nl = _offsets(bl)
    orr, nr = _offsets(br)
    T = np.zeros((nl, len(qn), nr))
    for (ql, s), blk in blocks.items():
        qr = ql + qn[s]
        T[ol[ql]: ol[ql] + bl[ql], s, orr[qr]: orr[qr] + br[qr]] = blk
    return T


def mps_to_vector(sites, bonds, qn):
    """Full state vector, site 0 most significant."""
    v = np.ones((1, 1))
    for j, blocks in enumerate(sites):
        T = dense_site(blocks, bonds[j], bonds[j + 1], qn)
        v = np.einsum("xa,asb->xsb", v, T).reshape(-1, T.shape[2])
    return v[:, 0]


def mpo_to_matrix(mpo):
    d = mpo.site.d
    T = np.ones((1, 1, 1))          # [row, col, w]
    for W in mpo.W:
        T = np.einsum("rcw,wstv->rsctv", T, W)
        r, s, c, t, v = T.shape
        T = T.transpose(0, 1, 2, 3, 4).reshape(r * s, c * t, v)
    return T[:, :, 0]


def left_matrix(sites, bonds, j, qn):
    """Dense [d^j, m_j] map of the left-block states defined by sites 0..j-1."""
    v = np.ones((1, 1))
    for k in range(j):
        T = dense_site(sites[k], bonds[k], bonds[k + 1], qn)
        v = np.einsum("xa,asb->xsb", v, T).reshape(-1, T.shape[2])
    return v


def right_matrix(sites, bonds, j, qn):
    """Dense [m_j, d^(L-j)] map of the right-block states defined by sites j..L-1."""
    L = len(sites)
    v = np.ones((1, 1))
    for k in range(L - 1, j - 1, -1):
        T = dense_site(sites[k], bonds[k], bonds[k + 1], qn)
        v = np.einsum("asb,by->asy", T, v).reshape(T.shape[0], -1)
    return v


def two_site_dense(psi, bl, br, qn):
    ol, nl = _offsets(bl)
    orr, nr = _offsets(br)
    d = len(qn)
    T = np.zeros((nl, d, d, nr))
    for (qa, s1, s2), blk in psi.items():
        qc = qa + qn[s1] + qn[s2]
        T[ol[qa]: ol[qa] + bl[qa], s1, s2, orr[qc]: orr[qc] + br[qc]] = blk
    return T


def embed_two_site(sites, bonds, j, psi, qn):
    """Full vector of the state whose bond-(j, j+1) wavefunction is psi."""
    Lm = left_matrix(sites, bonds, j, qn)
    Rm = right_matrix(sites, bonds, j + 2, qn)
    T = two_site_dense(psi, bonds[j], bonds[j + 2], qn)
    return np.einsum("xa,astc,cy->xsty", Lm, T, Rm).ravel()
