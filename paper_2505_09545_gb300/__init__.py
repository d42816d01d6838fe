"""GB300-native (sm_103a) Green's Dyadic Method hot path.

The compute lives in the CUDA library libgdm.so (C ABI: include/gdm.h); this
package only builds/loads it and marshals arguments (see `binding`)."""
from . import autograd  # noqa: F401
from .binding import (Context, GDMError, GDMProblem, alpha6_lorentz, assemble, autotune, autotune_batched, backward, cross_sections,
                      farfield, gpm_extract, incident_dipole, incident_gaussian, ldos, sigma_farfield, incident_planewave, lib, nearfield, nearfield_backward, padded_lda, residual,
                      solve, solve_batched, solve_gmres)

__all__ = ["Context", "GDMError", "GDMProblem", "alpha6_lorentz", "assemble", "autotune", "autotune_batched", "backward", "cross_sections", "farfield", "gpm_extract", "incident_dipole", "incident_gaussian", "ldos", "sigma_farfield", "incident_planewave",
           "lib", "nearfield", "nearfield_backward", "padded_lda", "residual", "solve", "solve_batched",
           "solve_gmres"]
