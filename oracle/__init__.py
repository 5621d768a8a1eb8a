"""CPU oracle for the two-site DMRG hot path -- TEST INFRASTRUCTURE ONLY.

A plain, slow, FP64 NumPy restatement of what the GPU engine computes, written from the
paper (Stoudenmire & White, "Real-Space Parallel Density Matrix Renormalization Group"):

* ``oracle.dmrg``     -- serial two-site DMRG (Sec. II, Eqs. wf and svd): the projected
                         Hamiltonian matvec L x W_i x W_{i+1} x R, Davidson, SVD truncation to
                         m states, gauge move, projected-operator (environment) updates.
* ``oracle.accsvd``   -- the Appendix's recursive accurate SVD.
* ``oracle.regions``  -- real-space parallel DMRG (Sec. II, Eqs. inverse, isvd, merge and
                         Fig. 4's staggered sweep), regions executed one after another.
* ``oracle.grad``     -- gradients of the projected-Hamiltonian application (reverse mode).
* ``oracle.icmps``    -- the inverse canonical gauge of Sec. IV (Lambda V Lambda at every bond)
                         and one-/two-site local expectation values in it.
* ``oracle.exact``    -- independent references: exact diagonalisation, the transverse-field
                         Ising free-fermion closed form, the AKLT energy.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may import
this package.  It shares no code with the CUDA engine; both read their inputs from the
``workloads`` module (seeded generators, no DMRG arithmetic).
"""
