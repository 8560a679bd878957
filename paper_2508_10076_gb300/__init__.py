"""GB300-native symmetric TensorMap contraction (libtk): permute, grouped sector GEMMs, scatter.

The compute path lives in the CUDA library ``_lib/libtk.so`` (built by :mod:`.build`), reached
through the C ABI declared in ``include/tk.h``; :mod:`.api` is the thin Python binding.  The
library is loaded on first use and loading fails loudly if it is missing (no fallback path).
"""

__all__ = ["build_library"]


def build_library(force: bool = False) -> str:
    from .build import build_library as _b
    return _b(force=force)
