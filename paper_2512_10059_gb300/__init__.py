"""GB300-native batched Boys-function evaluation (arXiv:2512.10059).

The compute path is libboys.so (hand-written sm_103a CUDA behind a C ABI,
declared in ``include/boys.h``); this package marshals torch CUDA tensors to
it.  Nothing here computes Boys functions on the host.
"""
from .api import (BoysFunction, RaggedPlan, boys, boys_eval, boys_eval_f32, boys_eval_fused,  # noqa: F401
                  boys_eval_host, boys_eval_ragged, boys_eval_ragged_noalloc, boys_pairwise,
                  boys_grad, kmax_limit, ragged_layout, ragged_noalloc_status, ragged_status, version)
