"""Packed layouts of the C ABI (include/pdmrg.h) <-> the oracle's dict-of-blocks tensors."""
import numpy as np


def psi_keys(bl, br, qn):
    keys = []
    for qa in bl:
        for s1 in range(len(qn)):
            for s2 in range(len(qn)):
                qc = qa + qn[s1] + qn[s2]
                if qc in br:
                    keys.append((qa, s1, s2))
    return keys


def pack_psi(psi, bl, br, qn):
    parts = [np.asarray(psi[k], np.float64).ravel() for k in psi_keys(bl, br, qn)]
    return np.concatenate(parts) if parts else np.zeros(0)


def unpack_psi(flat, bl, br, qn):
    out, off = {}, 0
    for (qa, s1, s2) in psi_keys(bl, br, qn):
        qc = qa + qn[s1] + qn[s2]
        n = bl[qa] * br[qc]
        out[(qa, s1, s2)] = np.asarray(flat[off: off + n]).reshape(bl[qa], br[qc])
        off += n
    return out


def env_keys(bond, flux):
    keys = []
    for q in bond:
        for w in range(len(flux)):
            if (q - int(flux[w])) in bond:
                keys.append((q, w))
    return keys


def pack_env(env, bond, flux):
    parts = []
    for (q, w) in env_keys(bond, flux):
        qk = q - int(flux[w])
        blk = env.get((q, w))
        parts.append((np.zeros((bond[q], bond[qk])) if blk is None else np.asarray(blk, np.float64)).ravel())
    return np.concatenate(parts) if parts else np.zeros(0)


def unpack_env(flat, bond, flux):
    out, off = {}, 0
    for (q, w) in env_keys(bond, flux):
        qk = q - int(flux[w])
        n = bond[q] * bond[qk]
        out[(q, w)] = np.asarray(flat[off: off + n]).reshape(bond[q], bond[qk])
        off += n
    return out


def random_env(bond, flux, rng):
    return {(q, w): rng.standard_normal((bond[q], bond[q - int(flux[w])])) for (q, w) in env_keys(bond, flux)}


def site_keys(bl, br, qn):
    return [(q, s) for q in bl for s in range(len(qn)) if (q + qn[s]) in br]


def pack_site(site, bl, br, qn):
    parts = [np.asarray(site[k], np.float64).ravel() for k in site_keys(bl, br, qn)]
    return np.concatenate(parts) if parts else np.zeros(0)


def unpack_site(flat, bl, br, qn):
    out, off = {}, 0
    for (q, s) in site_keys(bl, br, qn):
        n = bl[q] * br[q + qn[s]]
        out[(q, s)] = np.asarray(flat[off: off + n]).reshape(bl[q], br[q + qn[s]])
        off += n
    return out


def env_equal_support(a, b):
    """Keys with nonzero blocks in either dict."""
    return sorted(set(k for k, v in a.items() if np.any(v)) | set(k for k, v in b.items() if np.any(v)))
