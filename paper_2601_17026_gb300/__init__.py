"""GB300-native min-cut solver for proper-order multi-column graphs.

``pog``        thin binding of the C ABI (libpog.so, include/pog.h)
``autograd``   differentiable solve (quantise -> solve -> exact subgradient backward)
``synth``      seeded synthetic layered-horizon cost volumes
``autotune``   per-volume-class launch options (coordinate descent over timed solves), ``tuned.json``
``build``      nvcc build of libpog.so for sm_103a
"""
from .pog import (PogError, make_options, pog_backward, pog_build, pog_build_f32,  # noqa: F401
                  pog_build_f32_augmented, pog_energy, pog_export_state, pog_free, pog_maxflow, pog_quantise,
                  pog_solve_batch, pog_solve_batch_f32, pog_stats, pog_strerror, pog_surface, pog_surface_energy, solve)
