"""GB300 evaluation of Taylor-subtracted two-point correlators on grids of
complex p^2 (Windisch, Alkofer, Haase, Liebmann, arXiv:1205.0752).

The computation runs in libgfc (hand-written CUDA for sm_103a behind the C ABI
of include/gfc.h); this package only marshals arguments to it.
"""
from .binding import (GFC_F32X2, GFC_FP64, GFC_MIXED, EvalStats, GfcError, Router, Server, ServerStats,  # noqa: F401
                      angular_map, eval_grid, eval_points, eval_points_cond, eval_points_host, grid_points, last_stats,
                      library_path, load_library, make_grid, make_params, make_prop,
                      measure_pipe_peaks, region_map, release, version)
