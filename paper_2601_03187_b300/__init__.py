"""TaNG packet classification on B300 (sm_103a): Python binding of the C-ABI library libtang.so.

The binding only marshals arguments; rulesets, the network, the search, training and the
serving engine all run inside the library's CUDA kernels and C++ runtime.
"""
from ._native import (  # noqa: F401
    BF16, FP8, FP32, FUSED_N256, FUSED_PAIR, GRAPH, MEM_DEVICE, MEM_HOST, NO_MATCH, PATHS, Context, TangError, load_library, now,
    pack_model, unpack_model, LIB_PATH, EXPORTED, SEARCH_PAPER, checked_build, du_decide,
)
