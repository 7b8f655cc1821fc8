"""GB300-native finite-volume step for the shallow-water / shallow-moment hierarchy.

The compute path lives in the CUDA library ``libzoomy.so`` (C ABI declared in
``include/zoomy.h``); ``zoomy`` is its thin ctypes binding.  Importing this
package loads nothing: the library is opened on first use, and using it without
the compiled library raises instead of falling back to anything else.
"""
__all__ = ["zoomy", "inputs", "build"]
