"""FP64 CPU oracle for the matrix-free neo-Hookean Newton/Jacobi-PCG path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product (``paper_2104_13466_gb300``) never imports, links or
runs anything here, and this package imports nothing from the product.

The oracle is the plain definition of what the hot path computes, written in
numpy at float64 from Dias, Suzuki, Valente, Bittencourt (arXiv:2104.13466):

* ``quadrature``   Gauss-Legendre and Gauss-Lobatto-Legendre rules (Sec. 2).
* ``polynomials``  Jacobi and Lagrange polynomials (Sec. 2, eqs. lagrangian,
                   BasePadrao1D).
* ``basis1d``      standard nodal/modal 1D bases, simultaneous diagonalisation
                   (eqs. Diagonalizacao1-ParametroK) and minimum-energy
                   boundary modes (eqs. ExtensaoMEmassa-alphaKN).
* ``material``     neo-Hookean energy, second Piola-Kirchhoff stress and the
                   material tangent (Sec. 3, eqs. hyperelastic strain energy,
                   second Piolla_Kirchhoff relation).
* ``hexmesh``      structured box meshes, lattice numbering, Dirichlet faces.
* ``element``      dense tensor-product shape functions (eq.
                   ProdTensorialHexaedro) and element residual / tangent /
                   mass by direct quadrature loops (no sum factorisation).
* ``assembly``     global residual, sparse tangent, loads.
* ``solvers``      Jacobi-PCG, dense direct solve, Newton-Newmark step
                   (Sec. 4.2, eqs. newmark_acceleration, NR_explicit).
* ``manufactured`` fabricated-solution body forces and tractions (Sec. 5).
* ``adjoint``      vector-Jacobian product of the internal force and the
                   discrete adjoint of the explicit scheme (Sec. 4.1).
* ``condensation`` Schur complement on the element-interior modes (Sec. 4,
                   Sec. 5.1).
* ``quad``         plane-strain quadrilaterals (eq. ProdTensorialQuadrado).

Every function whose result is not pinned to something outside itself says
"parity unpinned" in its docstring; the tests in ``tests/test_oracle_*.py``
pin the rest.
"""
