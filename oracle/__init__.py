"""CPU FP64 oracle (test infrastructure only; see mca_oracle)."""
from .mca_oracle import *  # noqa: F401,F403
