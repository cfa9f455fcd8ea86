"""GB300 (sm_103a) modified-ziggurat generator (McFarland, arXiv:1403.6870).

The C ABI lives in include/zig.h and libzig.so; this package is its thin
Python binding.  Importing it loads the CUDA library and fails loudly if it
has not been built.
"""
from ._binding import *  # noqa: F401,F403
from ._binding import (ZigError, zig_build_tables, zig_exponential, zig_export_tables,  # noqa: F401
                       zig_normal, zig_set_fringe_limits, zig_status_poll, zig_strerror)
