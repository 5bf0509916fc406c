"""Measurement helpers: the thesis's effective-throughput metric and timing plumbing.

T_eff (thesis Art. 1, Section 2.3.2): A_eff = 2 D_unknown + D_known (Eq. 28), the bytes an
ideal solver must move per iteration (unknown DOFs read and written, known DOFs read);
T_eff = A_eff / t_it (Eq. 29). For the two-phase solver D_unknown = 12 N p and D_known = N p
(Eqs. 35-37: V (3), tau (6), Pt, Pf, phi unknown; one known field), so A_eff = 25 N p.
"""
from __future__ import annotations

import os
import shutil
import signal
import subprocess
import tempfile
import time

UNKNOWN_DOFS = 12
KNOWN_DOFS = 1


def a_eff_bytes(n_cells: int, p_bytes: int, unknown: int = UNKNOWN_DOFS, known: int = KNOWN_DOFS) -> float:
    """Effective main-memory access per iteration in bytes, Eqs. 28 and 35-37."""
    return float((2 * unknown + known) * n_cells * p_bytes)


def t_eff_gbs(n_cells: int, p_bytes: int, t_it_s: float, **kw) -> float:
    """Effective memory throughput in GB/s (1e9 bytes), Eqs. 29 and 38."""
    return a_eff_bytes(n_cells, p_bytes, **kw) / t_it_s / 1e9


class ClockSampler:
    """Samples nvidia-smi SM clocks and throttle reasons every 200 ms while active. start() returns
    once the first sample is written (or after 1 s), so the tool's start-up (driver queries) falls
    before the timed region that follows it."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int = 0):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self) -> None:
        if shutil.which("nvidia-smi") is None:
            return
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        self.proc = subprocess.Popen(
            ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
             "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        deadline = time.monotonic() + 1.0          # the tool may buffer its output: wait at most 1 s
        while time.monotonic() < deadline and self.proc.poll() is None and os.path.getsize(self.path) == 0:
            time.sleep(0.02)

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        self.proc.send_signal(signal.SIGTERM)
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.remove(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower().startswith("active")})
        sm = sorted(float(r[1]) for r in rows if r[1].replace(".", "").isdigit())
        smax = max((float(r[2]) for r in rows if r[2].replace(".", "").isdigit()), default=None)
        power = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": smax, "reasons": reasons,
                "samples": len(rows), "power_w_max": max(power) if power else None}


def rank_env() -> tuple[int, int, int]:
    """(rank, local_rank, world_size) from the torchrun environment (defaults 0, 0, 1)."""
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


def replica_seed(rank: int, base: int = 0) -> int:
    """Replicas-only scaling: rank r solves an independent instance with seed base + r."""
    return base + rank


def max_over_ranks(x: float, device=None) -> float:
    """Max of a scalar over all ranks of the default process group (identity without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())
