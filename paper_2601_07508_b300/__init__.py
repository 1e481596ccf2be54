"""mwmm: multiword modular matrix multiplication C = A B mod p on B300 (sm_103a).

The compute path lives in ``libmwmm.so`` (hand-written CUDA behind a C ABI);
``paper_2601_07508_b300.mwmm`` is the thin Python binding over it and is loaded
lazily so that ``paper_2601_07508_b300.inputs`` can be imported on machines
without a GPU or without the built library.
"""

__all__ = ["inputs", "mwmm"]
