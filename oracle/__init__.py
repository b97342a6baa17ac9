"""FP64 CPU oracle of the Microcosmos filament-fluid step.

TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
benchmark's CPU-baseline leg may import this package.  The product path (the
CUDA library and its Python binding) never imports it and shares no code with
it; the two sides meet only in the seeded input generators.
"""
from .mc_oracle import *  # noqa: F401,F403
