"""GB300-native greedy column subset selection (Farahat et al., arXiv:1312.6838).

The compute path is the C-ABI CUDA library libcss.so (include/css.h); this
package holds its build script, a ctypes binding and a torch front end.
"""
from . import _lib  # noqa: F401

__all__ = ["css", "build"]
