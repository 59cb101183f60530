"""B300-native (sm_103a) hot path of the RTU-grid lensing method (Enzi et al.).

The CUDA library and its ctypes binding load lazily (``from
paper_2606_30620_b300 import rtu``); importing the package itself loads
nothing, so the seeded input generators in ``inputs`` stay usable on hosts
without the built library.
"""
__all__ = ["inputs", "rtu"]
