"""CPU oracle for the PCG-ATKM solver -- TEST INFRASTRUCTURE ONLY.

Plain, slow, FP64 numpy/scipy restatement of the paper's method, used to
check the CUDA path.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import it; the product package never does,
and this package imports nothing from the product package.
"""
from .atkm_oracle import *  # noqa: F401,F403
