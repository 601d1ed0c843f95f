"""CPU FP64 oracle of the sparse-FFT hot path.  Test infrastructure only."""
from .sfft_oracle import *  # noqa: F401,F403
