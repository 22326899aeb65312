"""GB300-native shadow-sample evaluation of PV shading losses (3DPV method,
Robledo, Leloux & Lorenzo, arXiv 1410.5780).

* ``pv3d``    thin ctypes binding of the C ABI in include/pv3d.h (CUDA library)
* ``build``   compiles the CUDA library for sm_103a in-tree
* ``scenes``  seeded synthetic scenes, generators, sun tables and poses

The binding loads the compiled library lazily, on first use, and raises if it
is missing: there is no CPU path.
"""
__all__ = ["pv3d", "build", "scenes"]
