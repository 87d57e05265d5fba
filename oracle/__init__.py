"""FP64 CPU oracle of FastFCA-AS and conventional FCA.

TEST INFRASTRUCTURE ONLY: tests, the package smoke check and the benchmark's
CPU-baseline leg are the only users.  The CUDA library never imports it.
"""
from . import fastfca_as, fca  # noqa: F401
