"""GB300-native (sm_103a) sketching library: A_hat = S A with S regenerated
on the fly (arXiv 2310.15419), plus sketch-and-precondition least squares.

The compute path is libsketch.so (include/sketch.h); ``capi`` is its thin
binding.  Importing this package loads nothing: ``capi.load()`` builds (if
needed) and loads the library, and raises if that is impossible.
"""
__all__ = ["capi", "inputs", "build"]
