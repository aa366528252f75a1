"""GB300-native MGCG for interior-point and OC topology optimisation (Kocvara & Mohammed,
arXiv 1606.06201).

The compute path is the CUDA library ``libtopo_gb300.so`` built from ``csrc/``; the Python
modules here only marshal arguments to its C ABI (``include/topo.h``).  Importing this package
does not load the library; ``paper_1606_06201_gb300.topo`` does, and raises if it is missing.
"""
