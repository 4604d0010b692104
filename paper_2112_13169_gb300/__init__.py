"""GB300-native voxel-grid generation (arXiv 2112.13169).

The product is libvg.so (C ABI in include/vg.h, CUDA kernels in csrc/) and
the thin binding in `vg`.  Import `paper_2112_13169_gb300.vg` to use it.
"""
