"""ORACLE -- test infrastructure only.

Two independent checkers for the CUDA library, neither sharing code with it:

* ``estimator`` (``mcf_oracle.c`` through ctypes): the paper's estimators
  (Algorithm 3 RandFunmAction, Section 3.3 RandFunmDiag, Algorithm 2 RandFunm,
  Algorithm 1 classical MC) written as plain sequential C with its own
  Philox4x32-10.  Same seed -> same walks as the CUDA path, so the two agree up
  to floating-point summation order.
* ``reference``: the quantities the estimators converge to, in float64 --
  dense spectral evaluation on tiny graphs, truncated power series by repeated
  sparse products on large ones, and exact expectations/variances of the
  estimator by enumerating every walk (Lemma 2).

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  The library itself never does.
"""
from . import estimator, reference  # noqa: F401
