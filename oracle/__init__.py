"""Plain FP64 CPU oracle for the preconditioned spectral solves of variable-density flow.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and its Python
binding) imports, links or executes anything in this package; only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference`` legs of
``bench.py`` use it.

What it restates (Reynier et al., "A preconditioning for the spectral solution of
incompressible variable-density flows", arXiv 2403.06654):

* ``spectral``  -- periodic Fourier differentiation (the F-F-F discretisation of Sec. 3),
  a naive O(n^2) DFT written from the definition, the constant-density preconditioners
  (inverse Laplacian with the k=0 mode removed, Sec. 4.2 / Table 2 text; (I - a D^2)^-1,
  Eq. VDINSE.V).
* ``operators`` -- the pressure operator L_rho(phi) = div(rho^-1 grad phi)
  (Eq. VDINSE.Lrho / VDINSE.Lrho.num) and the variable-density viscous operator
  V_rho(u) = u - (dt/2) zeta(rho, u) (Eq. VDINSE.zeta, VDINSE.num.momentum.proj,
  1D form Eq. VDINSE.Vrho).
* ``solvers``   -- preconditioned CG, restarted GMRES and Richardson Minimal Residual
  (Sec. 3.1 list of solvers).
* ``step``      -- one semi-implicit second-order fractional step (Eqs. VDINSE.num.*).
* ``dense``     -- brute-force dense assembly on tiny grids (condition numbers, symmetry,
  null space), as in the condition-number study of Sec. 3.1 / 3.2.
* ``direct1d``  -- an exact, non-iterative solve of the 1D periodic pressure equation.

Everything is float64 numpy.  Transforms use ``scipy.fft`` (complex, all axes) as a library
primitive, single-threaded unless ``spectral.FFT_WORKERS`` is raised for timing on many
cores; the module also carries its own O(n^2) DFT written from the definition, used to pin it.

Parity pins: every function here is pinned by ``tests/test_oracle_*.py`` against closed
forms, exact solves, brute force or invariants (see the test module docstrings).
"""

from . import spectral, operators, solvers, dense, direct1d, step  # noqa: F401
