"""GB300-native certified interval bound propagation (IBP) of the soft-constrained
SC-DCOPF market-clearing objective over all N-1 line contingencies.

The compute path is the CUDA library ``_lib/libibp_gb300.so`` (sm_103a) behind
the C ABI of ``include/ibp.h``; this package is its thin Python binding.
"""
from . import _abi  # noqa: F401
from ._abi import IBPError, ibp_last_error  # noqa: F401
from .case import Case, algorithmic_flop, bound_multi, bound_multi_backward, dry_run_case  # noqa: F401

__all__ = ["Case", "IBPError", "dry_run_case", "algorithmic_flop", "ibp_last_error"]
