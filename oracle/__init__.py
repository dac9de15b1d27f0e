"""CPU reference ("oracle") for the wavelength-adaptive 27-point Helmholtz operator.

TEST INFRASTRUCTURE ONLY. Nothing on the product path imports this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may use it.  It shares no code with
the CUDA library (``paper_2108_08730_gb300``): it never imports it, and the
library never imports this.  Inputs come from the seeded generators in
``paper_2108_08730_gb300.synth``, which hold none of the method's arithmetic.

Everything here is plain, slow, complex128 NumPy/SciPy written from
Aghamiry, Gholami, Combe & Operto, "Accurate 3D frequency-domain seismic wave
modeling with the wavelength-adaptive 27-point finite-difference stencil"
(arXiv 2108.08730):

* ``weights``   -- dispersion relation (Eq. vtilde), linear form (Eq.
                   linear_basic), per-G fit (Eq. OPFD), joint fits (Eq.
                   eq_cost: G4, Gm) and the Tikhonov-regularised table
                   (Section 2.2, the minimise ||Hw-g||^2 + lam||Lw||^2 problem).
* ``pml``       -- complex stretching xi = 1 + i gamma/omega (Eq. 1.1-1.4).
* ``operator``  -- the row of [M + S] (Eqs. 3-8) assembled as scipy CSR.
* ``solve``     -- banded LU and dense LU of the assembled system.
* ``analytic``  -- homogeneous and constant-gradient Green's functions
                   (Section 3.1, the analytical references of benchmarks 1-2).
* ``multigrid`` -- textbook transfer operators and the damped-Jacobi sweep used
                   by the GPU preconditioner (not in the paper; definitions only).
* ``metrics``   -- relative L2 and the paper's l1 error (Eq. eqerror).

Parity status per function is stated in each module header; functions without
an independent pin say "parity unpinned".
"""
