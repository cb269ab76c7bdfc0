"""GB300-native SPH neighbour pipeline (arXiv 2005.02656, section 4).

The compute path is the CUDA library ``libsph.so`` (C ABI in include/sph.h),
built in-tree for sm_103a by ``_build.build()``.  ``SphSim`` keeps a particle
state in device memory (torch tensors) and drives the library; it raises if
the library is missing — there is no CPU path.
"""
from ._build import build  # noqa: F401


def __getattr__(name):
    if name in ("SphSim", "Params", "HostStepper", "measure_fp32_peak"):
        from . import sim
        return getattr(sim, name)
    if name == "Ensemble":
        from .ensemble import Ensemble
        return Ensemble
    if name in ("Rollout", "SphRolloutFn", "rollout"):
        from . import adjoint
        return getattr(adjoint, name)
    raise AttributeError(name)
