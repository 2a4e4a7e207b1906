"""FP64 CPU oracle (test infrastructure only; see pp_oracle)."""
from .pp_oracle import *  # noqa: F401,F403
from . import pp_oracle  # noqa: F401
