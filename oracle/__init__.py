"""Plain FP64 CPU oracle for the repeated-block SpMM method (arxiv 2508.06710).

TEST INFRASTRUCTURE ONLY.  Nothing in the library imports this package: only the tests,
the smoke check and the bench's CPU-baseline leg do.  It shares no code with the CUDA
path; the only module both sides use is ``workloads`` (seeded inputs, no arithmetic of
the method).

Contents, each function citing the passage of the paper it follows:
  * ``fvm``     staggered symmetry-preserving FVM operators M, G, L and the cell-to-face
                interpolator (Sec. 3, Eq. (ns); Sec. 4)
  * ``spmm``    SpMM over k right-hand sides (Sec. 2, Eq. (1) and Algorithm 1)
  * ``cg``      Jacobi-preconditioned CG per column, FP32-inner iterative refinement,
                batched uneven systems (Poisson solve of the projection method, Sec. 4)
  * ``stencil`` 13p and 27p Laplacians on uniform periodic grids (the denser patterns of Sec. 4.1)
  * ``refine``  coarse-to-fine prolongation and volume-weighted restriction of cell fields
                (inline mesh refinement, Sec. 3.3)
  * ``flow``    one Heun RK3 projection step of Eq. (ns) on m stacked flow states (Secs. 3, 4)
  * ``mg``      geometric-multigrid-preconditioned CG (V-cycle over 2:1 coarsenings; the
                multigrid preconditioning of Sec. 4 and Appendix A, built geometrically) and
                block CG over the k columns (Sec. 5.1)
  * ``mesh``    cotangent-weight Laplacian of a triangle mesh and its periodic extrusion
                (repeated geometries, Sec. 2; airfoil case, Sec. 4.3)
  * ``bounds``  arithmetic-intensity and speed-up models (Eqs. (ai), (pmspmm), (poipm), (pmite),
                (bbtilde), (fullpm); Appendix A)
  * ``unet``    FP64 forward/backward of the learned-initial-guess network

Parity status: every function is pinned by closed forms, invariants or brute force in
``tests/test_oracle_*.py`` except the trained network's predictions, whose parity is
unpinned (a learned heuristic); what is pinned there is that CG from the guess reaches
the same solution as CG from zero.
"""
