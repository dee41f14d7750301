"""Host-side runtime helpers: rank setup for one-process-per-GPU runs, the
barrier / max-over-ranks aggregation used by the benchmark, and an SM-clock
sampler. The hot path has no data exchange between GPUs (independent runs per
rank), so the only collectives are the barrier and the timing reductions."""
from __future__ import annotations

import os
import statistics
import subprocess
from dataclasses import dataclass


@dataclass
class Ranks:
    rank: int
    world: int
    local: int


def ranks_from_env() -> Ranks:
    return Ranks(int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
                 int(os.environ.get("LOCAL_RANK", "0")))


def init_dist(r: Ranks, backend: str):
    if r.world > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group(backend)


def barrier(r: Ranks):
    if r.world > 1:
        import torch.distributed as dist
        dist.barrier()


def aggregate(r: Ranks, seconds: float, units: float, device=None):
    """Max of `seconds` and sum of `units` over ranks: the whole-job time and
    work. Returns (max_seconds, total_units)."""
    if r.world == 1:
        return float(seconds), float(units)
    import torch
    import torch.distributed as dist
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    u = torch.tensor([units], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled while it runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: str, period_ms: int = 50):
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", str(period_ms), "-i", gpu],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None

    def stop(self, busy_mhz_floor: float = 0.0):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        load = [s for s in sm if s > busy_mhz_floor] or sm
        return {"sm_mhz": statistics.median(load), "sm_max_mhz": max(mx),
                "samples": len(sm), "reasons": sorted(reasons)}
