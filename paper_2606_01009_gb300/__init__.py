"""GB300-native MelT frontend: C-ABI library (libmelt.so) plus a thin ctypes binding.

``melt``   - the binding (same names as the C entry points in include/melt.h)
``inputs`` - seeded synthetic input generators (no method arithmetic)
"""
