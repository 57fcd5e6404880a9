"""GB300-native backward ray tracer for null geodesics in Kerr and tabulated
metrics (TARTARUS, arXiv 2609.08989): hand-written sm_103a CUDA behind the C ABI
in include/tartarus.h, with a thin ctypes binding.

Importing the package needs no GPU; the tracer entry points load
libtartarus.so on first use and raise if it cannot be built or loaded.
"""
from . import scenes  # noqa: F401
from . import tartarus  # noqa: F401

__all__ = ["scenes", "tartarus", "build"]


def build(force: bool = False) -> str:
    from . import _build
    return _build.build(force=force)
