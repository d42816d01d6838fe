"""CPU FP64 oracle for the GDM hot path: test infrastructure only (tests, smoke check,
benchmark CPU baseline). Shares no code with the CUDA library."""
from .gdm_oracle import *  # noqa: F401,F403
