"""CPU oracle for the MM method of fused lasso regression (TEST INFRASTRUCTURE).

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference
legs may import anything in this package.  The product path (the CUDA
library and its Python binding) never imports it, and the oracle imports
nothing from the product.  Inputs come from the flr_inputs package, which
holds no arithmetic of the method.

  oracle.mm     Eq. obj / pert / major / lin-sys and Algorithm 1 (dense
                Cholesky; Woodbury variant for large p)
  oracle.exact  exact special-case solvers that pin oracle.mm
"""
from . import mm, exact  # noqa: F401
