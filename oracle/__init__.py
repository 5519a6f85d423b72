"""Plain FP64 CPU oracle for the 2D acoustic PML wave operator and its time integrators.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and its Python
binding) may import, call or link anything in this package.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference arm use it.

It follows Ravelo, Schreiber & Peixoto, "High-order exponential integration for seismic
wave modeling" (arXiv 2401.16322):

* ``stencils``   -- Sec. 2.1 eqs. (spatial_8th_1/2), Appendix A free-surface rows, and
                    Fornberg's (1988) weight algorithm cited in Sec. 2.2.
* ``model``      -- Eq. (1)'s damping profile beta (Sec. 2) on the staggered grid of Fig. 1.
* ``operator``   -- the semi-discrete operator H of Eq. (1) (Sec. 2-2.2), matrix-free, plus
                    an independently assembled sparse H for small grids.
* ``source``     -- Ricker source term f and the augmented block [W; J] of Eq. (matrix_ampli).
* ``faber``      -- the Faber three-term recurrence of Sec. 3.2 and its coefficients.
* ``krylov``     -- the Arnoldi listing of Sec. 3.2 and a Pade matrix exponential.
* ``rk``         -- HORK (Sec. 3.2), RK3-2 and RK4-4 (Sec. 3.1).
* ``leapfrog``   -- the two-step scheme of Sec. 3.1.
* ``simulate``   -- time loops, receivers and the relative-L2 error measure.
* ``adjoint``    -- discrete adjoints of the Faber and HORK steps, the Krylov step's
                    linearisation, and the FWI misfit gradient.
* ``krylov_adaptive`` -- a KIOPS-style Krylov step with adaptive dimension and substeps
                    under an a-posteriori error estimate (the improvement Secs. 3.2 and 6 name).
* ``krylov_adjoint`` -- the exact discrete adjoint of the Krylov step (reverse mode through
                    Arnoldi and the small exponential) and the FWI gradient through it.
* ``leapfrog_adjoint`` -- the leap-frog step as a sparse linear map, its discrete adjoint and
                    the FWI gradient through it.
* ``wave3d``     -- the builder's 3D extension of Eq. (1) used by the 3D GPU passes.
* ``wave3d_pml`` -- a 3D PML with an auxiliary field that reduces exactly to Eq. (1).

Every floating-point quantity is IEEE double.  The module shares no code with the CUDA
path; the only module both sides import is the seeded input generator
(``paper_2401_16322_gb300.workloads``), which contains none of the method's arithmetic.

Parity status per function is stated in each module header; functions with no pin
other than themselves say "parity unpinned".
"""
