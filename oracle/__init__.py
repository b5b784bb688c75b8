"""FP64 CPU oracle of the AO real-time-control hot path (test infrastructure only).

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline / reference legs
may import this package; the CUDA product path never does.
"""
from .rtc_oracle import *  # noqa: F401,F403
from .rtc_oracle import OracleLoop, frame_slopes, quantize_rows, stored_matrix  # noqa: F401
