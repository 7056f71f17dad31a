"""GB300-native (sm_103a) mesh-vs-mesh intersection search.

Finds every intersecting triangle pair between two manifold meshes in R^4
(arXiv 2109.14814, Sec. 6): uniform-grid broad phase with bounding boxes, FP64
narrow phase solving the 4x4 system for (a, b, c, d), merged and sorted hits,
a batched form replayed from a CUDA graph, an FP64 adjoint, the damped-Newton
refinement of hits on the true surfaces (Sec. 7) and its continuation through
the family parameter (Sec. 8), and the method-of-layers sweep over half-layer
pairs (Sec. 5) as one batched search, and the FFT translation / derivative and
phase alignment of theta grids (Sec. 6.1, Sec. 7, Sec. 8.2).  All compute is
in libtms.so (C ABI in include/tms.h); this package only marshals arguments.
"""
from ._binding import (CONTINUE_STATUS, HIT_BYTES, REFINE_STATUS, STAGES, ContinueParams, Continued,
                       LayerPair, LayerSweep, layer_pairs, phase_align, theta_translate,
                       Refined, RefineParams, SurfacePair, continue_branches, refine, refine_params,
                       surface_pair, TMS_ERR_ARG, TMS_ERR_CAPACITY, TMS_ERR_CUDA,
                       TMS_ERR_STATE, TMS_ERR_TIMEOUT, TMS_OK, HitPoint, Hits, Mesh, Params, Stats,
                       TmsError, autotune, backward, last_error, last_patch_frames, last_stage_ms, last_stats,
                       lib, params,
                       probe_fp64_tflops, release_workspace, search, search_batched, search_host,
                       search_noalloc, status_str, version)

__all__ = ["CONTINUE_STATUS", "HIT_BYTES", "REFINE_STATUS", "STAGES", "ContinueParams", "Continued",
           "LayerPair", "LayerSweep", "layer_pairs", "phase_align", "theta_translate",
           "Refined", "RefineParams", "SurfacePair", "continue_branches", "refine", "refine_params",
           "surface_pair", "TMS_ERR_ARG", "TMS_ERR_CAPACITY", "TMS_ERR_CUDA",
           "TMS_ERR_STATE", "TMS_ERR_TIMEOUT", "TMS_OK", "HitPoint", "Hits", "Mesh", "Params",
           "Stats", "TmsError", "autotune", "backward", "last_error", "last_patch_frames", "last_stage_ms",
           "last_stats", "lib",
           "params", "probe_fp64_tflops", "release_workspace", "search", "search_batched",
           "search_host", "search_noalloc", "status_str", "version"]
