"""GB300-native cell-by-cell 3D Voronoi tessellation (votess method).

The computation runs in the CUDA library ``libvt.so`` (C ABI in
``include/vt.h``); :mod:`.api` is a thin PyTorch binding over it and
:mod:`.workloads` draws the seeded synthetic point clouds.
"""
from .cli import tessellate_numpy
from .api import (Batch, Cells, Params, VoronoiMoments, Workspace, batch_plan, clip_cells, emit, grid_build,
                  grid_resolution, knn, launch_count, lloyd, lloyd_step, probe_fma, moments_adjoint, tessellate, tessellate_batch,
                  tessellate_host, tessellate_stream, version, voronoi_moments, workspace_size)
from .tune import (autotune, autotune_batch, batch_cluster_index, cluster_class, cluster_index, default_space,
                   tuned_batch)

__all__ = ["Batch", "Cells", "Params", "VoronoiMoments", "Workspace", "batch_plan", "clip_cells", "emit",
           "grid_build", "grid_resolution", "knn", "launch_count", "lloyd", "lloyd_step", "probe_fma", "moments_adjoint", "tessellate",
           "tessellate_batch", "tessellate_host", "tessellate_stream", "version", "voronoi_moments", "workspace_size", "autotune",
           "autotune_batch", "batch_cluster_index", "cluster_class", "cluster_index", "default_space", "tuned_batch",
           "tessellate_numpy"]
