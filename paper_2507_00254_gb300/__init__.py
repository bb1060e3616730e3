"""GB300-native BP-SF decoder (arXiv 2507.00254): CUDA kernels behind a C ABI.

``bpsf`` is the ctypes binding of libbpsf (include/bpsf.h); ``codes`` builds
the benchmark codes through the library's builders; ``harness`` packs bits
and counts logical failures.  Build the library with ``build.build()``.
"""
from . import bpsf, codes, harness  # noqa: F401
from .bpsf import BpsfError, Decoder, Params, decode_multi  # noqa: F401
