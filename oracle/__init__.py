"""Plain, slow FP64 CPU oracle of the fully implicit phase-field method.

TEST INFRASTRUCTURE ONLY. Nothing in the product path may import it: only
``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline /
reference legs call it. It shares no code with the CUDA library; both sides
take their seeded inputs from ``synth``.

Layout (each function cites the passage of the paper it follows):

* ``fem``       Q1 elements on a structured box, 2-point Gauss rule (Sec. 2.1.1)
* ``residual``  the discrete residual F(U) of Eqs. (pf2), (conc2) with the
                theta-method of Eqs. (dpf)/(theta) at theta = 1, pure-metal and
                dilute-alloy variants; written for any numpy dtype so that a
                complex dtype gives complex-step derivatives
* ``jacobian``  J v, J^T w, dF/d eps4 and the sparse Jacobian by complex step
* ``precond``   the block-diagonal preconditioner of Eq. (pre) with the blocks
                of Eqs. (pref2)/(preconc2): assembly, point Jacobi and a
                geometric multigrid V-cycle with a Chebyshev smoother
* ``solver``    Newton with backtracking line search (Eqs. newton-update,
                glob, tolerance), forcing terms (Eqs. force1..forcing),
                restarted right-preconditioned GMRES with MGS, FD J v
                (Eqs. JFmatvec / preJFmatvec), and a direct-solve Newton
* ``adjoint``   discrete-adjoint gradient of the solid fraction through N steps

Every function is pinned by ``tests/test_oracle_*.py`` (textbook stencils,
flat interface, MMS convergence, conservation, symmetry, brute-force
Jacobians); none is "parity unpinned".
"""
