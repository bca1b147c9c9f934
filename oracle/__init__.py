"""CPU FP64 oracle of the explicit DG right-hand side (test infrastructure).

This package is test infrastructure only: the tests, the smoke check and the
benchmark's CPU-baseline / reference arm are the only callers.  The product
path (the CUDA library and its Python binding) never imports it, and it never
imports the product: the two share no code.  Inputs come from the seeded
generators in ``paper_2607_16044_b300.inputs`` (which hold none of the method's
arithmetic) or from plain arrays.

Contents (each function cites the passage of the paper it follows):

* ``basis``     -- Gauss-Legendre nodes/weights, Lagrange derivative matrix.
* ``geometry``  -- metric terms J, J d(xi_a)/dx and face area-normals.
* ``physics``   -- ideal-gas state, convective and viscous fluxes (Sec. 2),
                   local Lax-Friedrichs flux, adiabatic-wall states (App. B).
* ``residual``  -- the semi-discrete operator f(U) = -M^{-1} B(U) (Sec. 3.3,
                   Eq. for B_I, with the LLF/BR1 reading) and its BR1 gradient.
* ``ark``       -- the explicit ARK stage and solution updates (Sec. 4.2,
                   Algorithm 1) and the reverse (adjoint) stage recurrence.
* ``vjp``       -- vector-Jacobian products by reverse-mode differentiation of
                   the oracle, and dense Jacobians by the complex step.
* ``brute``     -- a dense, quadrature-based evaluation of the same weak form
                   used only to pin ``residual`` on tiny meshes.

Everything computes in float64 (or complex128 for the complex step).
Parity of the pieces that the paper does not itself fix (LLF, BR1, the wall
treatment for BR1, 3D) is pinned by invariants and closed forms in the tests
rather than by printed values: the paper prints no value of this operator.
"""
