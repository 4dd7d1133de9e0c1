"""GB300-native batched Boys-function evaluation (arXiv:2512.10059).

The compute path is libboys.so (hand-written sm_103a CUDA behind a C ABI,
declared in ``include/boys.h``); this package marshals torch CUDA tensors to
it.  Nothing here computes Boys functions on the host.
"""
from .api import boys_eval, boys_eval_fused, kmax_limit, version  # noqa: F401
