"""GB300-native batched unfolded ISTA / Step-LISTA / Oracle-ISTA for the Lasso
(arXiv 1905.11071).

The compute path is the CUDA library ``_build/libslista.so`` (C ABI in
``include/slista.h``); ``_lib`` binds its entry points under the same names,
``api`` allocates buffers and wraps them for torch users.  Importing this
package does not load the library; the first call does, and fails loudly if it
is missing.
"""
from ._lib import (  # noqa: F401
    SlistaError, PREC_FP32, PREC_TF32, PREC_BF16, PREC_BF16X3, PRECISIONS,
    FN_GRAM, FN_ISTA, FN_SLISTA_FWD, FN_SLISTA_BWD, FN_OISTA, FN_OBJECTIVE,
    slista_last_error, slista_device_status, slista_workspace_bytes, slista_ckpt_floats,
    slista_mask_words, lasso_gram, lasso_lipschitz, ista_forward, slista_forward, slista_backward,
    oista_forward, lasso_objective, slista_forward_noalloc, lista_forward, lista_workspace_bytes,
)
