"""GB300-native binary and run-length morphology with rectangular structuring
elements (Breuel, "Efficient Binary and Run Length Morphology and its
Application to Document Image Processing").

Submodules:
  * ``morph``  — Python binding of the C ABI in ``include/morph.h`` (loads
    ``libmorph.so``; raises if it is not built);
  * ``synth``  — seeded synthetic document pages (host C generator);
  * ``build``  — in-tree compilation of the native libraries.

Importing the package itself loads nothing native.
"""

__all__ = ["morph", "synth", "build"]
