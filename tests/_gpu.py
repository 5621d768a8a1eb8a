"""Helpers to drive the GPU engine from the shared workloads (no DMRG arithmetic here)."""
import numpy as np

import workloads as wl


def engine_for(pd, mpo, precision="fp64", kmax=8):
    W, flux, D = wl.pack_mpo(mpo)
    return pd.Engine(W, flux, D, list(mpo.site.qn), mpo.qtot, precision, kmax)


def load_mps(eng, mps, qn):
    data = np.concatenate([wl.pack_site(mps.sites[j], mps.bonds[j], mps.bonds[j + 1], qn)
                           for j in range(len(mps.sites))])
    eng.set_mps(mps.bonds, data)
