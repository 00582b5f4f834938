"""GB300-native (sm_103a) explicit Allen-Cahn stepper (arXiv 2105.09671).

The compute path is the CUDA library ``libac.so`` behind the C ABI of
``include/ac.h``; this package is its ctypes binding plus a PyTorch-facing
handle that allocates device memory.  There is no CPU fallback.
"""
from ._lib import (AC_ERR_CUDA, AC_ERR_INVALID, AC_ERR_NOMEM, AC_ERR_NONFINITE,  # noqa: F401
                   AC_ERR_TIMEOUT, AC_ERR_UNSUPPORTED, AC_F16S, AC_F32, AC_F64, AC_MAX_K, AC_OK,
                   AC_VARIANT_AUTO, AC_VARIANT_DIRECT, AC_VARIANT_STREAM, AC_TILE_AUTO, AC_NUM_TILES_3D, AC_NUM_TILES_2D,
                   AC_SHAPE_DUMBBELL, AC_SHAPE_STAR, AC_SHAPE_TORUS,
                   AcError, AcGridDesc,
                   EXPORTED, ac_autotune, ac_create, ac_destroy, ac_energy, ac_get_schedule,
                   ac_init_random, ac_init_shape, ac_init_sphere, ac_launch_count, ac_observe, ac_observe_noalloc, ac_phase_volume, ac_set_graph,
                   ac_set_schedule, ac_set_tile, ac_get_tile, ac_set_tune_cache, ac_status, ac_step, ac_version,
                   ac_workspace_bytes, lib,
                   lib_path, make_desc)


def __getattr__(name):
    # torch is imported lazily so that the binding loads without it
    if name in ("Simulation", "Batch", "DTYPES"):
        from . import sim
        return getattr(sim, name)
    raise AttributeError(name)
