"""GB300-native (sm_103a) implementation of the clotFoam species step.

The compute path is the CUDA library ``_build/libclot.so`` (sources in
``csrc/``, C ABI in ``include/clot.h``); this package is its thin Python
binding.  Importing works without a GPU; calling needs the built library and a
CUDA device and raises otherwise (there is no CPU fallback).
"""
from .binding import (CLOSED_ENDS, NO_ETA, NO_REACTION, NO_SIGMA, NO_TRANSPORT, NS, SPECIES,
                      ClotError, Ensemble, Fields, Fluxes, Mesh, Params, clot_device_status,
                      clot_diagnostics, clot_eta_solve, clot_eta_solve_noalloc, clot_profile_begin, clot_profile_end, clot_reaction_step, clot_species_step,
                      lib)

__all__ = ["Mesh", "Ensemble", "Fields", "Fluxes", "Params", "ClotError", "clot_species_step",
           "clot_reaction_step", "clot_eta_solve", "clot_diagnostics", "clot_device_status",
           "clot_profile_begin", "clot_profile_end", "clot_eta_solve_noalloc",
           "lib", "NS", "SPECIES", "NO_TRANSPORT", "NO_REACTION", "CLOSED_ENDS", "NO_ETA", "NO_SIGMA"]
