"""Float64 CPU oracle of the render path (test infrastructure only).

Only the tests, the smoke entry point and the benchmark's CPU-baseline leg may
import this package. The renderer never does."""
from .oracle import *  # noqa: F401,F403
