"""GB300 (sm_103a) Semi-Global Matching hot path of arXiv 1610.04121.

``paper_1610_04121_gb300.sgm`` is the ctypes binding of the C ABI in
``include/sgm.h``; importing it loads the CUDA library and fails loudly when
the library has not been built (``python -m paper_1610_04121_gb300.build``).
"""

__all__ = ["build", "sgm"]
