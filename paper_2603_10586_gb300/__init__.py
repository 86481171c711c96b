"""GB300-native QR-recursive compressed VIE solver for metasurfaces.

The compute lives in libvie.so (CUDA for sm_103a, C-ABI in include/vie.h);
``vie`` is its ctypes binding and ``build`` compiles it in-tree.
"""
from . import vie  # noqa: F401
