"""FP64 CPU oracle (test infrastructure only; never imported by the GPU library)."""
from .gw_oracle import *  # noqa: F401,F403
