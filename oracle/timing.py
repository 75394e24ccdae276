"""Wall-clock timing of the FP64 oracle on the host cores (the CPU baseline of the measured workloads).

ORACLE / TEST INFRASTRUCTURE: times the oracle as it stands (never tuned for this), one JSON
line per run: the workload, the grid, the RK3 steps timed (after one untimed warm-up step), the
threads used and the rate in cell-RK3-substeps/s = Nx Ny Nz 3 steps / seconds.  Full-size runs
use every host core; single-core runs use the full grid where that takes minutes and a stated
sample of the same physics and spacing where it would take most of an hour.

    python -m oracle.timing [--cores N] [--plan full|single|all]
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# (workload, grid override, steps) per plan; the grids of the three measured configurations
PLANS = {
    "full": [("taylor_green_32", {}, 20), ("cbl_256", {}, 10), ("les_512", {}, 3)],
    "single": [("taylor_green_32", {}, 20), ("cbl_256", {}, 1), ("les_512", dict(Nx=128, Ny=128, Nz=64), 1)],
}


def cpu_model() -> str:
    try:
        import subprocess
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                low = line.lower()
                if low.startswith("model name") or low.startswith("cpu part"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or platform.machine()


def time_run(workload: str, over: dict, steps: int, cores: int) -> dict:
    from oracle import oracle
    from paper_2502_14148_gb300 import inputs
    p = inputs.config(workload, **over)
    p["nthreads"] = cores
    m = oracle.OracleModel(p)
    m.set(**inputs.initial_state(p))
    m.project(1.0)
    m.time_step(p["dt"], 1)                       # warm-up step (page faults, thread start)
    t0 = time.perf_counter()
    m.time_step(p["dt"], steps)
    sec = time.perf_counter() - t0
    cells = p["Nx"] * p["Ny"] * p["Nz"]
    return {"workload": workload, "grid": f"{p['Nx']}x{p['Ny']}x{p['Nz']}", "full_size": not over,
            "steps": steps, "seconds": sec, "s_per_step": sec / steps, "threads": cores,
            "cell_substeps_per_s": cells * 3 * steps / sec}


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description="time the FP64 oracle on the host cores")
    ap.add_argument("--plan", choices=("full", "single", "all"), default="all")
    ap.add_argument("--cores", type=int, default=0, help="threads of the full-size plan (default: all)")
    a = ap.parse_args(argv)
    ncpu = os.cpu_count() or 1
    host = {"nproc": ncpu, "cpu": cpu_model(), "machine": platform.machine()}
    print(json.dumps({"host": host}), flush=True)
    plans = ["full", "single"] if a.plan == "all" else [a.plan]
    for plan in plans:
        cores = 1 if plan == "single" else (a.cores or ncpu)
        for workload, over, steps in PLANS[plan]:
            print(json.dumps(dict(time_run(workload, over, steps, cores), plan=plan)), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
