"""CPU FP64 oracle for SLaQ's stochastic Lanczos quadrature (test infrastructure).

This package is TEST INFRASTRUCTURE.  It is a plain, slow, obviously correct
NumPy/SciPy implementation of what the CUDA library computes, written from
the paper (Tsitsulin, Munkhoeva, Perozzi, "Just SLaQ When You Approximate",
WWW'20).  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline /
reference legs of ``bench.py`` may import it.  The product path (the C-ABI
library and its Python binding) never imports, links or runs anything here,
and this package shares no code with the CUDA sources.

Modules and the passages they follow
------------------------------------
``laplacian``  Sec. 2: L = D - A and the normalized Laplacian
               I - D^{-1/2} A D^{-1/2}; the density matrix P = L / tr(L)
               of Sec. 2.1.
``probes``     Sec. 3.1 (Eq. trace): zero-mean, unit-variance probe vectors,
               Rademacher signs from a SplitMix64 counter-based generator.
``lanczos``    Sec. 3.1: s-step Lanczos giving the tridiagonal T = Q^T L Q,
               with one classical Gram-Schmidt pass against all previous
               Lanczos vectors after the three-term update; and Lanczos with
               partial reorthogonalization (Simon's omega-recurrence; not in
               the paper), which reorthogonalizes only when the estimated
               loss of orthogonality passes sqrt(eps).
``quadrature`` Eq. quadratic and Eq. slq, Algorithm 1: eigh(T) gives nodes
               theta and weights tau^2 (first eigenvector components);
               Hutchinson mean over probes.
``descriptors`` Eq. heat-trace (NetLSD heat trace), the wave trace, and the
               VNGE of Definition 1 / Sec. 2.1.
``exact``      the plain definitions through a dense eigendecomposition
               (the ground truth the paper compares against, Sec. 4.1).
``distance``   spectral distances between descriptors (Sec. 4.2).
``variance``   the polynomial control variate of Sec. 3.1 ("2-term
               polynomial" variance reduction) and tr L^2.

Every function is pinned by ``tests/test_oracle_*.py`` against closed forms,
invariants and the worked example of Fig. 1; nothing here is unpinned.
"""

from . import laplacian, probes, lanczos, quadrature, descriptors, exact, distance, variance  # noqa: F401
