"""FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY.

Plain, slow, obviously correct implementations of what the GPU library
computes: the paper's compensation + planar RMA with exact transforms
(``rma.rma_exact``), the same with high-accuracy fast Gaussian gridding
(``rma.rma_fast``), and direct back-projection (``bpa.bpa``).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA
library and never imports it; both sides take their inputs from ``synth``.
"""
from . import bpa, rma  # noqa: F401
from ._native import build  # noqa: F401
