"""GB300-native syndrome decoding of CSS quantum LDPC codes (normalized min-sum BP, arXiv 2508.07879).

Modules
-------
``qldpc``      ctypes binding of libqldpc.so (C ABI in include/qldpc.h): Graph, decode,
               decode_pair, decode_host.  Importing it loads the CUDA library or raises.
``workloads``  seeded synthetic codes (HGP, lifted product, bivariate bicycle) and error samplers.
``gf2``        GF(2) rank / logical-operator checks used to score decoder outputs.
``build``      compiles libqldpc.so for sm_103a.

The decoder names (``Graph``, ``decode``, ...) are re-exported lazily so that importing the
package for its input generators does not load the CUDA library.
"""
from __future__ import annotations

__version__ = "0.1.0"

_LAZY = {"Graph", "decode", "decode_pair", "decode_host", "QldpcError"}


def __getattr__(name):
    if name in _LAZY:
        from . import qldpc
        return getattr(qldpc, name)
    raise AttributeError(name)
