"""FP64 CPU oracle for the single-node boundary schemes of Zhao & Yong (arXiv:1712.08288).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and its
Python binding) may import, call or link anything from this package.  It exists so
that the tests, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / reference arm
of ``bench.py`` can check and time the GPU path against a plain, slow and obviously
correct restatement of the paper.

Layout
------
``lattices``  velocity sets, weights, MRT matrices (Appendix; D3Q19 from the
              d'Humieres et al. 2002 polynomial basis the Appendix cites).
``adjoint``   reverse-mode (discrete adjoint) of ``lbm`` for a velocity-mismatch
              loss; gradients with respect to S, per-link q and wall velocity
              (single-node scheme).
``lbm``       one lattice-Boltzmann step: MRT collision (Appendix), equilibrium
              Eq. (42), advection Eq. (2.2b), the boundary scheme Eq. (2.13) built
              from Eqs. (2.5)-(2.7) and (2.9) in the paper's order (optionally the
              two-node variant of Remark (2), Eq. 2.11), moments and the relative L2
              error of Sec. 3.1.

Everything is float64 numpy; dense matrices, two population arrays (pre- and
post-collision), push streaming.  No blocking, fusion or reordering beyond what the
equations state.

Parity status: every function here is pinned by a ``-m "not gpu"`` test
(``tests/test_oracle_*.py``) against printed tables, closed forms, textbook special
cases or invariants.  The only quantitative results the paper prints are the
matrices M and the statement that the observed orders are close to 2; its convergence
plots are not available, so the oracle's absolute error values are not pinned to the
paper (only their order of convergence is).
"""

from . import adjoint, lattices, lbm  # noqa: F401
