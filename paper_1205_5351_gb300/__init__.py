"""GB300-native TILT by LADMAP with warm starts (Ren & Lin, arXiv 1205.5351).

The solver lives in a C-ABI shared library (``csrc/``, declared in ``include/tilt.h``);
``paper_1205_5351_gb300.tilt`` is its ctypes binding.  Importing the package itself loads
nothing."""
__version__ = "0.1.0"
