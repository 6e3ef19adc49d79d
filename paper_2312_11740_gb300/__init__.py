"""GB300-native variable-density pressure-Poisson solve (arXiv 2312.11740 hot path).

Thin Python binding over the C-ABI in include/mp_poisson.h: the functions
below carry the C names and only marshal arguments (torch tensors for
device memory and streams).  Every step of the solve runs in the CUDA
library; there is no CPU path.
"""
from .poisson import (  # noqa: F401
    MPError,
    Poisson,
    mp_opts_default,
    mp_poisson_apply,
    mp_poisson_destroy,
    mp_poisson_divergence,
    mp_poisson_get_components,
    mp_poisson_get_fields,
    mp_poisson_get_profile,
    mp_poisson_get_stats,
    mp_poisson_project,
    mp_poisson_project_step,
    mp_poisson_project_step_host,
    mp_poisson_rhs,
    mp_poisson_rhs_noalloc,
    mp_poisson_set_geometry,
    mp_poisson_set_mass_flux,
    mp_poisson_deflated_energy,
    mp_poisson_set_opts,
    mp_poisson_set_profiling,
    mp_poisson_setup,
    mp_poisson_solve,
    mp_status_str,
)
from .net import Net, mp_conv3d_fwd, mp_conv3d_wgrad, mp_poisson_set_net  # noqa: F401
