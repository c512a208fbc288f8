"""Plain FP64 CPU oracle for the exponential-DG hot path (test infrastructure).

This package is test infrastructure, not product code.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline / reference legs of
``bench.py`` may import it.  It shares no code with the CUDA library in
``paper_2011_01316_gb300/``: it does not import that package, and that
package never imports this one.

Everything here is written for a reader checking it against the paper
(Kang & Bui-Thanh, "A scalable exponential-DG approach for nonlinear
conservation laws", arXiv 2011.01316):

* ``lgl``         - Legendre-Gauss-Lobatto nodes, weights and the nodal
                    differentiation matrix (textbook formulas; LGL quadrature
                    is the paper's choice, Sec. 4).
* ``dg``          - the collocated nodal DG operator R(q) and the frozen-flux
                    linear operator L(q~)v for Burgers (Sec. 3.1, Eq. BurgerL /
                    BurgerN with the Lax-Friedrichs fluxes) and the Euler
                    equations (Sec. 3.2, Eq. euler-split-3dd, with the local
                    Lax-Friedrichs flux the paper adopts for Euler in Sec. 5.1).
* ``expm``        - dense matrix exponential by scaling and squaring of a
                    truncated Taylor series.
* ``krylov``      - the phi-function sum of Eq. (linear_combination_of_phifunctions)
                    by Arnoldi on the augmented matrix (Sec. 2.3), with
                    sub-stepping and a recorded decision trace.
* ``integrators`` - the EPI2, EXPRB32 and EXPRB42 steps (footnotes of Sec. 5).

Every function states the passage it follows.  Where the paper is silent the
reading taken is stated in the docstring.  Parity status: every function is
pinned by the tests in ``tests/test_oracle_*.py``; none is "parity unpinned".
"""

from . import lgl, dg, expm, krylov, integrators  # noqa: F401
