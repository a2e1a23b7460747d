"""CPU oracle (test infrastructure only).

Plain, slow, single-threaded reference for the 3D distance and 3D intersection
operators of arxiv 1808.09571 (Sec. 3.2.2, Sec. 3.2.3, Eqs. 3-4), the exact
mesh volume of Eq. 2 (volume.py), plus an FP64 reference of the proposal
network.  Only the test suite, the smoke check and
the CPU-baseline leg of the benchmark may import this package; the product
path never does, and this package imports nothing from it.
"""
from .oracle import (  # noqa: F401
    build, lib, orient3d, orient2d, tri_intersects, tri_feature_d2, tri_distance,
    pt_tri_d2, seg_seg_d2, pt_seg_d2, mesh_distance_brute, mesh_intersects_brute,
    mesh_distance_pruned, mesh_intersects_pruned, batch_pruned,
)
