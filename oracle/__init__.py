"""FP64 CPU oracle for the Fourier transform on SU(2) (Delgado & Umana).

TEST INFRASTRUCTURE ONLY.  Only the test-suite, the package smoke check and
the benchmark's CPU-baseline / reference legs may import or run anything in
this package.  The product path (the CUDA library and its Python binding)
never imports it, and this package imports nothing from the product path.

What it computes (all in float64 / complex128):

* ``grid``        -- Euler-angle sampling grid (Sec. 4, Definition of the
                     sampling grid) and the packed coefficient layout.
* ``quadrature``  -- beta-node weights: Clenshaw-Curtis on x_k = cos(beta_k)
                     and the paper-literal Riemann weights sin(beta_k)*pi/(N-1).
* ``basis``       -- matrix coefficients t^l_{mn}(u) from the derivative
                     definition (Sec. 3, Theorem), P^l_{mn} in exact rationals
                     from the Rodrigues-type formula (Sec. 3), and Wigner-d
                     values by the three-term recurrence (Sec. 4, Lemma on the
                     Legendre recurrence and its Jacobi analogue).
* ``transform``   -- the forward transform as the direct O(N^6) quadrature sum
                     (Sec. 5) and as the separated O(N^4) form (Sec. 4,
                     Proposition on the factorised Riemann sum; Sec. 6); the
                     synthesis (Sec. 3, Peter-Weyl expansion) and the adjoint.
* ``shifted``     -- the shifted Legendre polynomials A_r^L, B_r^L and the
                     divide-and-conquer projections of Sec. 4 (Theorem
                     "Divide-and-conquer"), used as identities in tests.
* ``pool``        -- runs ``transform``'s row-restricted routines across the
                     host cores (spawned processes) for large bandwidths.

Parity status: every function here is pinned by tests in ``tests/`` against
closed forms, library routines (scipy), exact rationals or invariants.
"""
from . import grid, quadrature, basis, transform, shifted  # noqa: F401
