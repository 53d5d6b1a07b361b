"""GB300-native block-sparse matrix multiply and tensor contraction (DBCSR hot path).

The compute path is the C-ABI library ``libbst.so`` (hand-written CUDA for sm_103a),
declared in ``include/bst.h`` and bound here with ctypes (``paper_1910_13555_gb300.bst``).
Importing this package does not load the library; the first call into ``bst`` does,
and it raises if the library is missing -- there is no CPU fallback.
"""
__all__ = ["bst", "workloads"]
