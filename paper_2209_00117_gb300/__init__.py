"""GB300-native (sm_103a) jump flooding for dynamic Voronoi diagrams.

Implements the hot path of "GPU Voronoi Diagrams for Random Moving Seeds"
(Stevenson-Regla and Navarro): JFA and dynamic JFA frames over an int32 label
map, in hand-written CUDA kernels behind the C ABI of ``include/vd.h``.

Importing the package loads nothing; :mod:`paper_2209_00117_gb300.vd` loads
``_build/libvd.so`` on first use and raises if it is missing.
"""

__all__ = ["vd", "inputs", "build"]
