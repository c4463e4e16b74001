"""GB300-native cylindrical-grid SART (Goethals, Heyndrickx, Boone, arXiv 2005.11976).

The reconstruction path lives in the CUDA library ``libcylct.so`` (sources in ``csrc/``,
C ABI in ``include/cylct.h``); :mod:`.cylct` is its thin ctypes binding.  Importing this
package does not load the library; :func:`.cylct.load` does, and raises if it is missing.
"""
__all__ = ["cylct", "synth"]
