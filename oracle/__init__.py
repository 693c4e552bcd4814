"""FP64 CPU oracle of the periodic compressible-Euler finite-volume method of arXiv:2512.13403.

TEST INFRASTRUCTURE ONLY.  Nothing in the product (the CUDA library and its Python binding)
imports, calls or links anything here; only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may.  The GPU path shares no code, table or constant generator
with this package.

The oracle is plain PyTorch on the CPU in float64: whole-array operations written in the
order the paper gives them, with no blocking or fusion, so each function can be checked
against the cited section or equation by eye.  Modules:

  hydro      primitive recovery, MUSCL/MC reconstruction, HLLC, unsplit RHS, RK2, CFL dt,
             conserved totals                                    (Sec. 3, App. A)
  forcing    Ornstein-Uhlenbeck forcing with its counter-based Gaussian draws (Sec. 3.1.1)
  cooling    optically thin cooling, trapezoid / subcycled update with floor   (Sec. 4.3)
  multigrid  7-point Poisson operator, red-black Gauss-Seidel V-cycle, gravity source (Sec. 5.2)
  driver     one full step in the order hydro -> forcing -> gravity -> cooling
  adjoint    vector-Jacobian product of the step by reverse-mode autodiff of this oracle
  corrector  residual 3D CNN corrector with BF16 operands and periodic padding (Sec. 7)

Parity status of each function is stated in its module header; "parity unpinned" marks the
ones with no independent pin.
"""
