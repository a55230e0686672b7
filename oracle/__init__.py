"""Plain FP64 CPU oracle for the PF-MP HMC hot path (Haar, Kamleh, Zanotti, Nakamura,
"Applying polynomial filtering to mass preconditioned Hybrid Monte Carlo").

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this package: only
``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` use it.  It shares no code with the CUDA library; the only module
both sides take inputs from is ``pfmp_inputs`` (seeded random numbers, no arithmetic of
the method).

Everything is written as the plain definition with PyTorch CPU tensors in float64 /
complex128, vectorised over lattice sites with ``torch.roll`` shifts and ``einsum``
contractions.  There is no blocking, fusing or reordering beyond what each definition
states.  Derivatives with respect to the gauge links (the force terms of App. C) are
taken by ``torch.autograd`` of the bilinear forms the paper writes down; that library
derivative plays the role a library matmul plays elsewhere.

Modules
  lattice     geometry, boundary shifts, gamma matrices, su(3) generators, exp map
  dirac       clover field, Wilson hop, full M, even-odd Schur complement M-hat, K, J
  solvers     CG, batched CG on normal equations for complex shifts, dense solves
  cheby       Chebyshev roots / normalisation / residues (App. A, App. C)
  action      gauge action, PF-MP action terms, heatbath, forces (App. C); the general
              term list (filter, factorised filter, filter correction, Hasenbusch
              ratio, inverse) and the paper's schemes 1PF, 2PF, 1MP, 2MP, PF-MP,
              2PF-1MP, 1PF-2MP
  spectrum    extreme eigenvalues of K (dense), Lanczos tridiagonal and its Ritz values
              (App. A: the filter ellipse must enclose the spectrum)
  integrator  2MN / leapfrog step arrays, generalised multi-scale merge (App. B),
              MD trajectory and Metropolis test (Sec. 2.1), for PF-MP and for a
              general term list

Parity status: every function is pinned by a ``-m "not gpu"`` test against a closed
form, an invariant, brute force or a value the paper prints, except the clover-term
sign convention (the paper is Wilson-only), which is pinned only through Hermiticity,
gauge covariance and finite differences of the action -- "parity unpinned" for the
physical sign of c_sw.
"""
