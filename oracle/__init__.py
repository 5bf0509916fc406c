"""Plain FP64 CPU oracle of the PT + Picard porosity-wave solver — TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this package. The CUDA product path never imports, links or runs it, and the two share
no code: this package compiles ``pt_oracle.c`` with the host C compiler and calls it through
ctypes, on plain numpy arrays in the natural staggered shapes (see ``pt_inputs.field_shapes``).

What it computes: thesis Art. 1, Eqs. 17-27 on the staggered grid of Fig. 1, one PT iteration
per call of ``iteration`` and one physical time step per ``step`` (details in pt_oracle.c).
Parity unpinned for the thesis's own numbers (it prints no field values); the oracle is pinned
by closed forms, invariants and a brute-force Newton solve in the tests.
"""
from .binding import (  # noqa: F401
    build, lib_path, OracleParams, OracleRes, State, make_state, init_viscosities,
    begin_step, iteration, iterate_n, end_step, step, system_residual, coefficients, darcy,
    divergence, stress, momentum, advection, tau_II, ORACLE_OK, ORACLE_EINVAL,
    ORACLE_ENOTCONV, ORACLE_ENAN, max_threads,
)
