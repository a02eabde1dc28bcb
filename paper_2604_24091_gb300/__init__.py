"""GB300-native (sm_103a) rejection-free vacancy AKMC on bcc Fe-Cu-Ni-Mn.

The compute path is libakmc.so (CUDA kernels behind the C ABI in
include/akmc.h); this package only marshals arguments to it.
"""
from .akmc import (AkmcError, Batch, SelectPlan, select_logits, load_library, last_error,  # noqa: F401
                   workspace_bytes, OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, ETRAPPED, ENUMERIC, STATUS_NAMES)
