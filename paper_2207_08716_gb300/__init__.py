"""GB300-native pseudo-transient (PT) + Picard solver for 3-D nonlinear poroviscoelastic
two-phase flow (porosity waves; thesis arxiv 2207.08716, Art. 1).

The compute path is the CUDA library ``libpt_gb300.so`` (sources in ``csrc/``, C ABI in
``include/porowave_pt.h``); this package builds it (``native.build_library``) and calls it
through ctypes (``solver.PTSolver``). There is no CPU fallback.
"""
from .native import build_library, load  # noqa: F401

__all__ = ["build_library", "load"]
