"""GB300-native integral-direct J/K build by Rys quadrature (arXiv 2407.09700).

The compute path is liberi.so (CUDA, sm_103a) behind the C-ABI in include/eri.h;
``eri`` is its thin ctypes binding.
"""

from .build import build  # noqa: F401
from .eri import (  # noqa: F401
    ERI_FP64, ERI_MIXED, ERI_WANT_J, ERI_WANT_K, EriError, Plan, load_library, probe_fma_peak, rys_roots,
    header_symbols, one_electron, Batch, check_class_tables, check_density,
)
