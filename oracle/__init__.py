"""FP64 CPU oracle for the linearized Boltzmann solver (Wu, Zhang, Liu, Zhang, Reese,
"A fast iterative scheme for the linearized Boltzmann equation", arXiv:1612.04488).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this package: only
``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` use it.  It shares no code, tables or constants with the CUDA
library; both sides build their own tables from the formulas.

Plain, slow and written for reading against the paper:

* ``velocity``  -- velocity grid and the equilibrium VDF (Sec. 2, first equation).
* ``fsm``       -- hard-sphere linearized collision operator (Eq. LBE_collision) by the
                   fast spectral method, plus two independent evaluations used as pins
                   (explicit spectral convolution, brute-force velocity quadrature).
* ``transport`` -- second-order upwind transport sweeps (Eq. LBE_iteration), 1D plates
                   and 2D rectangular ducts, diffuse walls.
* ``solver``    -- CIS (Eq. LBE_iteration) and SIS (Eqs. syn_LBE, first_order,
                   diffusion_LBE, guided, with the N-penalty of Sec. 2.5 footnote).
* ``eig``       -- Fourier-mode eigenvalue analysis (Sec. 2.3, Eqs. conv_iteration,
                   acceleratred_iteration).
* ``mixture``   -- binary hard-sphere mixture (Sec. 4): the four linearized collision
                   operators in a dense spectral form, the viscosity that fixes delta, and
                   the SIS of Eqs. LBE2_true1 / LBE2_true2 for plates.

Every floating-point quantity is float64.  Parity status of each function is stated in
its module docstring; functions without an independent pin say "parity unpinned".
"""
