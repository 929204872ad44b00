"""Plain FP64 CPU oracle for the surrogate-matrix IGA wave path.

TEST INFRASTRUCTURE ONLY. Nothing in the product path imports this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may call it.

The oracle is written directly from the paper (Drzisga, Keith, Wohlmuth,
"The surrogate matrix methodology: accelerating isogeometric analysis of
waves", arXiv:2004.05197) in the paper's order and notation:

* ``bspline``    - open uniform knot vectors, Cox-de Boor B-splines, Gauss-Legendre
                   (Sec. 3.1; element-loop Gauss quadrature of Sec. 5.1)
* ``geometry``   - geometry maps F and wave-speed coefficients c (Eq. weakforms,
                   Eq. LinearWaveEnergy)
* ``assembly``   - true stiffness K and mass M by element-loop quadrature
                   (Eq. weakforms, Eq. SurrogateEoM, Eq. KeyIdentity)
* ``surrogate``  - sampling (Sec. 5.1), B-spline interpolation of the stencil
                   functions (Sec. 3.3) and the symmetric / kernel-preserving
                   surrogate matrices (Eq. DefinitionOfSurrogateMatrixSymmetric,
                   Eq. DefinitionOfSurrogateMatrixSymmetricKernel)
* ``wave``       - Jacobi-preconditioned CG on the consistent mass and leapfrog
                   time stepping of M u'' + K u = f (Sec. 4.6 context); the CG start
                   of each step (polynomial extrapolation in time, ``cg_start``)
* ``adjoint``    - receiver misfit and its tangent-linear directional derivative
                   with respect to the wave speed's B-spline coefficients
* ``multipatch`` - several patches glued along sides with a first-visit global
                   numbering (Sec. 3.2 / 3.4 multi-patch remarks)

Every routine is deliberately slow and unblocked; numpy / scipy routines are used
only as library primitives (dense solves, sparse mat-vecs, eigensolvers).
"""
