"""Plain, slow FP64 CPU oracle of the Nystrom-accelerated primal LS-SVM ODE solver.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call or
execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` use it.  It shares no code with the CUDA path
(``paper_2510_04094_gb300``) and imports nothing from it.

Modules
-------
``core``     RBF kernel and its t-derivatives (Section 3, Eq. 9 and the two
             derivative formulas after it), the Nystrom factor (Appendix A.3),
             explicit features (eq32), the linear primal system of Lemma 1
             (Section 3.1, proof in Appendix A.4) and its solve.
``newton``   Lemma 2 (Section 3.2, Eq. 2.2, proof in Appendix A.5):
             the nonlinear KKT system F = grad L = 0 solved by Newton's method
             (Eq. 3.2.1), dense (m+n+p) Jacobian for small n and the exactly
             equivalent reduced (y-eliminated) form for large n.
``dual``     Checks only: the dual LS-SVM of the same ODE problem with the
             Nystrom kernel (exact equivalence) and with the true RBF kernel
             (classical LS-SVM of Appendix A.1 / Mehrkanoon et al.).
``adjoint``  Gradient of a loss on the fitted solution with respect to the ODE
             coefficients, the initial values and sigma, by complex-step
             differentiation of an equivalent kernel-coordinate solve.

Every function states the passage it follows.  Where the paper is silent or
garbled, the reading taken is stated in the docstring.

Parity status: all functions here are pinned by ``tests/test_oracle_*.py``
(closed forms, the accuracy figures of the paper's table in Appendix B.7, exact identities,
finite differences, brute-force minimisation); none is "parity unpinned"
except the Duffing accuracy against the true solution, which has no closed form
(the oracle's Duffing Newton iterate is pinned only through its KKT conditions).
"""

