"""GB300-native (sm_103a) implementation of the clotFoam species step.

The compute path is the CUDA library ``_build/libclot.so`` (sources in
``csrc/``, C ABI in ``include/clot.h``); this package is its thin Python
binding.  Importing works without a GPU; calling needs the built library and a
CUDA device and raises otherwise (there is no CPU fallback).
"""
from .binding import (CLOSED_ENDS, DEVIATION, HEUN, MLP_ENGINE_MMA, MLP_ENGINE_TCGEN05, MLP_NPARAM, NO_ETA, NO_REACTION, NO_SIGMA,
                      NO_TRANSPORT, NS, SPECIES, STRANG, SYNC_STATUS, WALL_LAGGED,
                      ClotError, Ensemble, Fields, Fluxes, Mesh, Mlp, Params, clot_device_status,
                      clot_diagnostics, clot_diagnostics_async, clot_eta_solve, clot_eta_solve_noalloc, clot_profile_begin,
                      clot_profile_end, clot_reaction_step, clot_species_step, clot_surrogate_forward,
                      clot_species_step_surrogate, clot_surrogate_grad, clot_surrogate_infer, clot_surrogate_pairs,
                      clot_surrogate_train, clot_surrogate_workspace, lib)

__all__ = ["Mesh", "Ensemble", "Fields", "Fluxes", "Params", "Mlp", "ClotError", "clot_species_step",
           "clot_reaction_step", "clot_eta_solve", "clot_diagnostics", "clot_diagnostics_async", "clot_device_status",
           "clot_profile_begin", "clot_profile_end", "clot_eta_solve_noalloc",
           "clot_surrogate_pairs", "clot_surrogate_forward", "clot_surrogate_workspace", "clot_surrogate_grad",
           "clot_surrogate_train", "clot_surrogate_infer", "clot_species_step_surrogate",
           "lib", "NS", "SPECIES", "MLP_NPARAM", "MLP_ENGINE_MMA", "MLP_ENGINE_TCGEN05", "NO_TRANSPORT", "NO_REACTION", "CLOSED_ENDS", "NO_ETA",
           "NO_SIGMA", "SYNC_STATUS", "HEUN", "STRANG", "WALL_LAGGED", "DEVIATION"]
