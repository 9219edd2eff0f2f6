"""GB300-native condensed interior-point method for AC optimal power flow.

The hot path -- model derivatives, G_x refactorisation, multi-right-hand-side
triangular solves, the dense condensed matrix, its Cholesky factor and the
step recovery -- is CUDA (sm_103a, FP64) behind the C ABI of include/condipm.h;
``binding`` is its thin ctypes wrapper.
"""
from .binding import Handle, OPFError, load_library  # noqa: F401
