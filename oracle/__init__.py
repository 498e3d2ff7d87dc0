"""FP64 CPU oracle of the SGL transform.  Test infrastructure only: imported by
tests, the smoke check and the CPU-baseline leg of the benchmark, never by the
library."""
from .sgl_oracle import *  # noqa: F401,F403
