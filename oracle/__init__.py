"""FP64 CPU oracle for one time step of the low-Mach flame-sheet solver.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product path (``paper_2603_01727_gb300``) never imports it, and it
imports nothing from the product path: the two share no code.

The oracle is a plain, slow, literal restatement of the method of Severino,
Fachini, Gennaro, Rodriguez & Souza, "Numerical method for strongly
variable-density flows at low Mach number: flame-sheet regularisation and a
mass-flux immersed boundary method" (arXiv 2603.01727):

* ``operators``  -- interpolation, difference and integration operators (Eqs 3.20-3.22)
* ``flame``      -- regularised flame-sheet state relation (Eqs 3.34-3.42, 2.49-2.50)
* ``boundary``   -- ghost-cell boundary conditions (Eqs 3.43-3.46, 3.27-3.28)
* ``ibm``        -- shifted mask, penalisation targets and mass source (Eqs 3.30-3.33, 4.19-4.21)
* ``poisson``    -- exact solve of the compact pressure Poisson equation (Eqs 3.9, 3.17, 3.24)
* ``step``       -- predictor-corrector step (Eqs 3.1-3.19, 3.23-3.26)
* ``convergence``-- observed order and GCI (Eqs 4.1-4.3)
* ``stretched``  -- the tanh grid map (Eq 4.18) and 1D non-uniform operators
  (Eqs 3.20-3.24) used to check the stretched path of ``operators``
* ``objective``  -- integrated heat release (the adjoint's objective)

Everything is float64 numpy; the only library primitives used as steps are the
FFT / DCT of ``scipy.fft`` (Poisson solve on a uniform grid), the sparse LU of
``scipy.sparse.linalg`` (Poisson solve on a stretched grid), a bracketing root
finder of ``scipy.optimize`` (the alpha of Eq 4.18) and dense linear algebra of
``numpy.linalg`` (brute-force checks).  There is no blocking, fusion or
reordering beyond what the equations state.
"""

from . import operators, flame, boundary, ibm, poisson, step, convergence, stretched  # noqa: F401
