"""GB300-native velocity fixed-point iteration (V-FPI) contact solver.

The solver itself is the CUDA library ``libvfpi`` (C-ABI declared in
``include/vfpi.h``); :mod:`paper_2201_09212_gb300.vfpi` is its thin ctypes
binding and :mod:`paper_2201_09212_gb300.scenes` generates seeded inputs.
Importing this package does not load the library.
"""
__version__ = "0.1.0"
