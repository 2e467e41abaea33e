"""FP64 CPU oracle for TILT by LADMAP with warm starts.  Test infrastructure only: it may
be imported by the tests, by ``__graft_entry__.smoke()`` and by the CPU-baseline leg of
``bench.py``, and by nothing else."""
from .tilt_oracle import *  # noqa: F401,F403
