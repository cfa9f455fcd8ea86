"""GB300 (sm_103a) modified-ziggurat generator (McFarland, arXiv:1403.6870).

The C ABI lives in include/zig.h and libzig.so; this package is its thin
Python binding.  The binding (and with it libzig.so) loads on first use of
any API name and raises ImportError if the library has not been built:
there is no CPU fallback.  `paper_1403_6870_gb300.build` compiles it.
"""
import importlib

_binding = None


def __getattr__(name):
    global _binding
    # only API names load the binding; anything else (e.g. the `build`
    # submodule) falls through to the normal import machinery
    if not (name.startswith(("zig_", "ZIG_", "Zig")) or
            name in ("raw_call", "LIB_PATH", "pack_requests", "request_dtype")):
        raise AttributeError(name)
    if _binding is None:
        _binding = importlib.import_module("._binding", __name__)
    try:
        return getattr(_binding, name)
    except AttributeError:
        raise AttributeError(f"module {__name__!r} has no attribute {name!r}") from None
