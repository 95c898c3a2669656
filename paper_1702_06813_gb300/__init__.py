"""GB300-native RenderMap pose-cost engine (Ryde & Ding, arXiv 1702.06813).

The map is a labelled triangle mesh of the free/occupied/unknown interfaces (Sec. IV.A); a
pose is scored by rendering the map's z-buffer from it and comparing it per pixel with an
observed range image by Table I (Sec. IV.B, Eq. 1). All of it runs in hand-written sm_103a
CUDA kernels behind the C ABI of include/rendermap.h; this package is the thin binding.
"""
from .rendermap import (OUTCOMES, RM_PINHOLE, RM_RAYTABLE, Intrinsics, Map, RenderMapCost,  # noqa: F401
                        Scan, align, align_batch, blur_scan, cost, cost_grad, cost_grad_batch,
                        cost_grad_vertices, cost_params, cost_sweep, depth_normals, dfo_align, dfo_params,
                        icp_align, icp_align_batch, icp_terms, meshify, pose_from_x, pose_retract, render_depth,
                        twist_grad,
                        scan_from_range, sequential_icp)
from ._native import RenderMapError, exported_symbols  # noqa: F401
