"""CPU oracles for the PCG-ATKM solver -- TEST INFRASTRUCTURE ONLY.

Two independent plain, slow, FP64 restatements of the paper's method, used to
check the CUDA path: ``oracle.atkm_oracle`` in numpy/scipy (re-exported
here) and ``oracle.cpp_oracle``, a C++17 program with its own FFT and
Faddeeva function (built by ``oracle.cpp_oracle.build``).  Only ``tests/``,
``__graft_entry__`` (build and smoke) and the CPU legs of ``bench.py`` may
import them; the product package never does, and this package imports
nothing from the product package.
"""
from .atkm_oracle import *  # noqa: F401,F403
