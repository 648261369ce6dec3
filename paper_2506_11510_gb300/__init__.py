"""tetvol for GB300: path tracing of heterogeneous media on adaptive tetrahedral
grids built by longest-edge bisection (Benyoub & Dupuy, SIGGRAPH Talks 2025).

The computation lives in libtetvol.so (CUDA, sm_103a, C ABI in include/tetvol.h);
this package builds it in-tree and binds it with ctypes.
"""
from .api import (Batch, Grid, GridInfo, build_scene_grid, grid_import, grid_render, grid_trace_paths, leb_build, leb_rebuild,
                  rebuild_scene_grid,
                  new_stats, release_build_memory, stats_dict, tet_optical_depth, tet_render, tet_render_ext, tet_trace_ext_paths,
                  tet_trace_paths)
from ._native import TetvolError
from . import cache
from .cache import RadianceCache

__all__ = ["Batch", "Grid", "GridInfo", "TetvolError", "build_scene_grid", "grid_import", "grid_render", "grid_trace_paths",
           "leb_build", "leb_rebuild", "rebuild_scene_grid", "new_stats", "release_build_memory", "stats_dict", "tet_optical_depth", "tet_render", "tet_trace_paths", "tet_render_ext", "tet_trace_ext_paths", "cache",
           "RadianceCache"]
