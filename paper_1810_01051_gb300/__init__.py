"""GB300 multi-pattern Rabin-Karp matcher (Shah & Oza, arXiv 1810.01051).

``rk`` is the ctypes binding of the C-ABI library ``lib/librk.so``;
``matcher.Matcher`` is a small convenience wrapper that takes device buffers
from PyTorch.  Build the library with ``build_lib.build()``.
"""

from . import rk  # noqa: F401
from .rk import (  # noqa: F401
    RkError, rk_build, rk_destroy, rk_table_info, rk_workspace_bytes, rk_scan_device,
    rk_sort_device, rk_search_device, rk_search, rk_window_hashes_device, unpack_keys,
)
