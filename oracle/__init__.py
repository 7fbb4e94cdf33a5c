"""FP64 CPU oracle for monitored free-fermion trajectories (arXiv 2508.18468).

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, obviously correct
restatement of what the GPU path computes.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference arm may
import it.  The CUDA library never calls into it and shares no code with it:
the only common element is the counter-based Philox4x32-10 generator, which
each side implements separately from its published definition (Salmon,
Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11).

Modules
-------
philox      Philox4x32-10, the uniform and normal draws built on it.
lattice     hopping matrix (Sec. II; 2d in Sec. IV), propagator exp(-i H dt),
            Neel / checkerboard initial orbitals (App. A).
trajectory  one time step of the projective (App. A, Eqs. (A1)-(A2)) and
            homodyne / QSD (App. A, Eq. (A4)) protocols on the L x N orbital
            matrix U, Householder re-orthonormalisation (App. A).
observables entanglement entropy (Sec. II), mutual information (Sec. IV),
            density-density correlation C(r) (Eq. (2)).

Every function works in float64 / complex128.
"""
