"""FP64 CPU oracle (test infrastructure only; see fj_oracle's header)."""
from .fj_oracle import *  # noqa: F401,F403
