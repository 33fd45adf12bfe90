"""GB300-native cell-by-cell 3D Voronoi tessellation (votess method).

The computation runs in the CUDA library ``libvt.so`` (C ABI in
``include/vt.h``); :mod:`.api` is a thin PyTorch binding over it and
:mod:`.workloads` draws the seeded synthetic point clouds.
"""
from .api import (Cells, Params, Workspace, clip_cells, emit, grid_build, grid_resolution, knn, launch_count,
                  tessellate, tessellate_host, version, workspace_size)

__all__ = ["Cells", "Params", "Workspace", "clip_cells", "emit", "grid_build", "grid_resolution", "knn",
           "launch_count", "tessellate", "tessellate_host", "version", "workspace_size"]
