"""GB300-native random batch Ewald (RBE) k-space path.

The computation lives in ``librbe.so`` (CUDA for sm_103a, C ABI in ``include/rbe.h``);
this package holds its build step and a ctypes binding.  ``inputs`` holds the seeded
synthetic workloads.  Importing the package does not load the library; the first call
does, and raises if it cannot be built or loaded.
"""
from ._binding import (  # noqa: F401
    RBE_OK, RBE_EINVAL, RBE_ENOMEM, RBE_ECUDA, RBE_ETIMEOUT, RBE_ENONFINITE, RBE_ESAMPLE, RBE_ESTATE,
    RBE_FP64, RBE_FP32_PHASE, RBE_RHO_FP64, RBE_RHO_COMP32, RBE_RHO_FP32,
    RBEError, Context, load, library_path,
    rbe_create, rbe_destroy, rbe_set_stream, rbe_set_precision, rbe_set_box, rbe_sample_k,
    rbe_kspace_forces_virial, rbe_kspace_forces_virial_host, rbe_kspace_forces_virial_xyzq, rbe_kspace_weighted, rbe_get_rho, rbe_sync,
    rbe_version, rbe_set_kernel_timing, rbe_get_kernel_times, rbe_measure_pipe, rbe_sample_k_noalloc,
    NptParams, System, NptReplica, rbe_npt_init, rbe_npt_step, RBE_CELL_DOUBLES,
    WaterParams, water_params, WaterReplica, rbe_water_init, rbe_water_step, CELL_EXCL,
    FlexParams, FlexSystem, FlexReplica, rbe_flex_init, rbe_flex_step, RBE_FLEX_CELL_DOUBLES,
    FLEX_H, FLEX_PH, FLEX_W, FLEX_KT, FLEX_PT, FLEX_EK, FLEX_EC, FLEX_EL, FLEX_V, FLEX_HAM, FLEX_STEP, FLEX_BUILDS, Server, ServerConfig, Request, piston_mass,
    piston_masses_rect, RBE_BAROSTAT_NONE, RBE_BAROSTAT_ISO, RBE_BAROSTAT_ANISO, RBE_BAROSTAT_SEMI, CELL_PC,
    CELL_WD, CELL_K2D, CELL_PD, Batch, BatchItem,
    rbe_set_seed, rbe_set_sampler, rbe_set_pressure_batch, rbe_set_sample_reuse, RBE_SAMPLER_EXACT, RBE_SAMPLER_OFFLINE, RBE_SAMPLER_MH,
)
