"""CPU oracle for the voxel-grid generation method (arXiv 2112.13169).

Test infrastructure only: the tests, the smoke check and the benchmark's
CPU-baseline leg are its only users.  The CUDA library never imports it.
"""
from .oracle import Oracle, OracleGrid, OracleParams, default  # noqa: F401
