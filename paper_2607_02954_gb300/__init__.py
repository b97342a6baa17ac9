"""GB300-native filament-fluid step of Microcosmos (arXiv 2607.02954).

The compute path is libmc.so (hand-written sm_103a CUDA kernels behind the C
ABI of include/mc.h); this package holds its ctypes binding, the Python API
and the seeded synthetic-world generators.  The library is loaded on first
use and its absence is an error.
"""
from .synth import Params, WorldSpec  # noqa: F401


def __getattr__(name):
    if name in ("World", "Server", "step_batched", "default_params", "stream_handle", "autotune", "launch_config",
                "set_launch_config"):
        from . import world
        return getattr(world, name)
    raise AttributeError(name)
