"""geo3d: exact 3D distance and 3D intersection between triangle meshes on
GB300 (sm_103a), after arxiv 1808.09571 (Sec. 3.2.2, Sec. 3.2.3).

The compute path is the CUDA library libgeo3d.so (C ABI in include/geo3d.h);
this package holds its in-tree build, a ctypes binding and the seeded
synthetic geometry generators.  Importing it loads nothing; the library is
loaded on first use and its absence is an error, never a fallback.
"""
from ._build import build as _build_lib


def build(force: bool = False) -> str:
    """Compile libgeo3d.so for sm_103a in-tree; returns its path."""
    return _build_lib(force=force)


def __getattr__(name):
    if name in ("Context", "Mesh", "MLP", "G3DError", "load", "declared_functions", "OP_DISTANCE",
                "OP_INTERSECTS", "G3D_F32", "G3D_F64", "library_path", "linestring_mesh", "collection_mesh"):
        from . import geo3d
        return getattr(geo3d, name)
    raise AttributeError(name)
