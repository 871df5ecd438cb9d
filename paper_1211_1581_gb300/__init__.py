"""GB300-native FP64 and FP64-accurate dense matrix product (EuroBen mod2am,
Sec. 3.1: c_ij = sum_k a_ik b_kj).

The compute path is the C-ABI library ``libmxm.so`` (hand-written sm_103a
CUDA); ``paper_1211_1581_gb300.mxm`` is its thin Python binding.  Importing
this package does not load the library; the first call does, and fails
loudly if it is missing.
"""
__all__ = ["inputs", "mxm"]
