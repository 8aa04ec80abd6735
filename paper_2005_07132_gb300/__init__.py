"""GB300-native fKK-EC (factorised Kramers-Kronig with phase- and scale-error
correction, arXiv 2005.07132).

The compute lives in libfkk.so (C ABI: include/fkk.h), hand-written CUDA for
sm_103a; this package is its thin Python binding (`_lib`), the in-tree build
(`build`) and the seeded synthetic input generator (`synth`).  Importing the
package does not load the library; the first binding call does, and raises
if the library has not been built.
"""
from ._lib import Context, FkkError, kk_per_spectrum, lib  # noqa: F401

__all__ = ["Context", "FkkError", "kk_per_spectrum", "lib"]
