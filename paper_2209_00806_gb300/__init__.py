"""GB300-native TBPM: Chebyshev-Bessel propagation of random states under a
sparse tight-binding Hamiltonian, the correlation C(t) and the DOS
(arXiv 2209.00806, Sec. 2.2 and 2.4), as hand-written sm_103a CUDA kernels
behind the C ABI of ``include/tbpm.h``.

``_native`` is the ctypes binding with the C names; ``tbpm`` adds a small
object wrapper.  Importing fails loudly if the CUDA library is not built.
"""
from . import _native  # noqa: F401  (raises ImportError when libtbpm.so is missing)
from ._native import (TBPM_FP32, TBPM_FP64, TbpmError, tbpm_bessel_coefficients,  # noqa: F401
                      tbpm_dos)
from .tbpm import Propagator, ac_conductivity, dos, dos_adjoint, fermi_coefficients  # noqa: F401
