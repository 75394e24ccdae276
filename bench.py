#!/usr/bin/env python
"""Benchmark: cell-RK3-substeps/s of the nonhydrostatic Boussinesq RK3 step.

Workload (default ``les_512``): 512 x 512 x 256 cells, FP32, WENO9 advection,
Smagorinsky-Lilly closure, T and S with a linear EOS, f = 1e-4, surface stress
and heat flux, dt = 2 s, seeded synthetic initial state.  A "step" is one full
RK3 step (three substages of closure + fused tendency + pressure projection).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank advances its own replica on its own GPU (the
single-domain LES has no data-parallel split without halo and transpose
exchanges); the value is the aggregate over ranks.  The model state (1.3 GB)
is larger than L2, so no L2 flush is needed between steps.  One JSON line is
printed by rank 0.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0
SMS, FP32_LANES, SM_MAX_MHZ = 152, 128, 2070.0
CPU_SAMPLE = dict(Nx=128, Ny=128, Nz=64)     # bounded oracle sample, same spacing and physics
CPU_SAMPLE_1CORE = dict(Nx=64, Ny=64, Nz=64)  # the single-core oracle sample


# ------------------------------------------------------------------ algorithmic counts
def weno_flops(r: int) -> int:
    """Floating-point operations of one WENO(2r-1) reconstruction as the method states it
    (an FMA counts 2): r substencil dot products (2r^2), r smoothness quadratic forms evaluated
    as sum_a t_a (sum_{b>=a} C_ab t_b) (r(r+1) + 2r each), WENO-Z weights (tau: 2; per
    substencil: +eps, reciprocal, ratio, square+1, times d: 6), sum of weights (r), weighted sum
    (2r), final normalisation (2)."""
    return 2 * r * r + r * (r * (r + 1) + 2 * r) + 2 + 6 * r + r + 2 * r + 2


def tendency_flops_per_cell(p: dict) -> int:
    """Algorithmic FP operations of the fused tendency + RK update per cell (one substage)."""
    r = (p["weno_order"] + 1) // 2
    P = r - 1
    nt = len(p["tracers"])
    nrec = 9 + 3 * nt                       # 3 momentum components x 3 directions + tracers x 3
    flops = nrec * weno_flops(r)
    flops += 9 * 3 * P                      # centered advecting velocities (symmetric form)
    flops += nrec                           # flux = velocity x reconstruction
    flops += (3 + nt) * 9                   # flux divergence: 3 differences + 3 scaled sums per field
    closure = p.get("closure", "none")
    if closure in ("smagorinsky", "amd"):
        flops += 9 * 11 + 3 * nt * 5         # eddy stress fluxes (edge averages, strain, flux) + tracer fluxes
    elif closure == "scalar":
        flops += nrec * 3
    flops += 2 * 5                          # Coriolis
    flops += 2 * 4 + 6                      # hydrostatic pressure gradient + column integral
    flops += (3 + nt) * 4                   # RK3 update
    return flops


def substep_bytes_per_cell(p: dict) -> int:
    """Algorithmic HBM bytes of one RK3 substage per cell: (4n + 9) words, n = 3 + tracers
    (state in, G^{m-1} in, G^m out, state out; projection: read u~ for div, write the spectrum,
    tridiagonal read/write, inverse read/write, read p for the correction)."""
    n = 3 + len(p["tracers"])
    w = 4 if p.get("precision", 32) == 32 else 8
    return (4 * n + 9) * w


FALLBACK_BF16_TFLOPS = 1900.0


def measured_peaks() -> dict:
    try:
        with open(MEASURED_PEAKS) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured", "sm_max_mhz": float(d.get("sm_max_mhz", SM_MAX_MHZ)),
                "bf16_tflops": float(d.get("bf16_tflops", FALLBACK_BF16_TFLOPS)),
                "bf16_tflops_sustained": float(d.get("bf16_tflops_sustained", FALLBACK_BF16_TFLOPS))}
    except Exception:
        return {"hbm_gbs": FALLBACK_HBM_GBS, "source": "fallback", "sm_max_mhz": SM_MAX_MHZ,
                "bf16_tflops": FALLBACK_BF16_TFLOPS, "bf16_tflops_sustained": FALLBACK_BF16_TFLOPS}


# the closure network: 32 -> 128 -> 128 -> 128 -> 16, two flops per multiply-add
MLP_FLOPS_PER_SAMPLE = 2 * (32 * 128 + 128 * 128 + 128 * 128 + 128 * 16)


PROFILED_SOURCES = {"tendency": ["tendency_kernel.cuh", "weno_coeffs.h", "tendency_f32_r5.cu", "tendency_f32_r5_smag.cu",
                                 "ocn_internal.cuh"],
                    "mlp_closure": ["mlp.cu", "column.cuh"]}


def source_hash(kernel: str) -> str:
    """sha256 (first 16 hex digits) of the sources a profiled kernel is compiled from."""
    h = hashlib.sha256()
    for name in PROFILED_SOURCES[kernel]:
        h.update(open(os.path.join(ROOT, "paper_2502_14148_gb300", "csrc", name), "rb").read())
    return h.hexdigest()[:16]


def profiled_field(kernel: str, workload: str, key: str):
    """A number from the committed ncu summary of a kernel, valid only while the kernel source
    hash recorded there matches the current sources (else None)."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.txt")
    try:
        fields = {}
        for line in open(path):
            if ":" in line:
                k, v = line.split(":", 1)
                fields[k.strip()] = v.strip()
        if fields.get("source_sha256_16") != source_hash(kernel):
            return None
        return float(fields[key].split()[0])
    except Exception:
        return None


def profiled_traffic(kernel: str, workload: str):
    """DRAM bytes per full-size launch from the committed ncu summary (None when stale)."""
    return profiled_field(kernel, workload, "dram_bytes_per_full_launch")


def tendency_bytes_per_cell(p: dict, first_substage: bool = False) -> int:
    """Algorithmic HBM bytes of the fused tendency + RK update per cell: the state in and out, G^m
    out and G^{m-1} in (not in an RK3 first substage, zeta = 0), nu_e out when it is computed in
    the kernel (FP32 Smagorinsky-Lilly) or in with the other closures."""
    n = 3 + len(p["tracers"])
    w = 4 if p.get("precision", 32) == 32 else 8
    words = 3 * n + (0 if first_substage else n)
    if p.get("closure") in ("smagorinsky", "amd"):
        words += 1
    return words * w


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs (our own child process)."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.rows = []
        self.proc = None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(index)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) == 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        if not self.rows:
            return None
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


# ------------------------------------------------------------------ distributed (replicas)
def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl"
        try:
            import torch
            if not torch.cuda.is_available():
                backend = "gloo"
            else:
                torch.cuda.set_device(local)
        except Exception:
            backend = "gloo"
        dist.init_process_group(backend=backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------ oracle legs
def oracle_rate(workload: str, steps: int, warmup: int = 0, cores: int = None, sample=CPU_SAMPLE, keep=None):
    """Time the FP64 oracle (as it stands) on the bounded sample with `cores` threads (default:
    all host cores); returns (cell-substeps/s, s/step, cores, sample description).  `keep` (a
    dict) receives the sample's parameters and the oracle model after the timed steps."""
    from oracle import oracle
    from paper_2502_14148_gb300 import inputs
    cores = cores or os.cpu_count() or 1
    p = inputs.config(workload, **sample)
    p["nthreads"] = cores
    m = oracle.OracleModel(p)
    m.set(**inputs.initial_state(p))
    m.project(1.0)
    if warmup:
        m.time_step(p["dt"], warmup)
    t0 = time.perf_counter()
    m.time_step(p["dt"], steps)
    dt = time.perf_counter() - t0
    cells = p["Nx"] * p["Ny"] * p["Nz"]
    if keep is not None:
        keep.update(params=p, model=m, steps=warmup + steps)
    return cells * 3 * steps / dt, dt / steps, cores, f"{p['Nx']}x{p['Ny']}x{p['Nz']} cells of the {workload} physics and spacing, {steps} RK3 step(s), FP64 oracle"


def run_reference(args, world, rank):
    if rank != 0:
        return 0
    from paper_2502_14148_gb300 import inputs
    p = inputs.config(args.workload)
    rate, sps, cores, sample = oracle_rate(args.workload, args.steps, args.warmup)
    line = {"metric": "cell-RK3-substeps/sec", "value": rate, "unit": "cell-substeps/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": sps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": workload_desc(p), "sample": sample},
            "cpu_baseline": {"value": rate, "unit": "cell-substeps/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": rate, "unit": "cell-substeps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def workload_desc(p: dict) -> str:
    return (f"{p['name']}: {p['Nx']}x{p['Ny']}x{p['Nz']} FP{p['precision']}, WENO{p['weno_order']}, {p['closure']}, "
            f"tracers {','.join(p['tracers'])}, f={p.get('f', 0)}, dt={p['dt']} s")


# ------------------------------------------------------------------ our arm
def size_override(args) -> dict:
    if not args.size:
        return {}
    nx, ny, nz = (int(x) for x in args.size.lower().split("x"))
    return dict(Nx=nx, Ny=ny, Nz=nz)


def run_ours(args, world, rank, local):
    import numpy as np
    import torch
    from paper_2502_14148_gb300 import build, inputs, ocn

    if rank == 0 or world == 1:
        build.build()
    barrier(world)
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    p = inputs.config(args.workload, **size_override(args))
    cells = p["Nx"] * p["Ny"] * p["Nz"]
    st = inputs.initial_state(p, seed=inputs.SEED + rank)
    model = ocn.Model(p, device=dev)
    model.set(**st)
    dt = p["dt"]
    qab2 = args.stepper == "qab2"

    def configure(m):
        if qab2:
            m.set_time_stepper("qab2", 0.1)
        if args.vertical != "none":
            # a surface-intensified vertical diffusivity profile (boundary-layer-like), same for momentum and tracers
            zf = np.asarray(p["z_faces"])
            prof = 1e-2 * np.exp((zf - zf[-1]) / 32.0)
            m.set_vertical_diffusivity(prof, prof, implicit=(args.vertical == "implicit"))

    configure(model)
    substeps = 1 if qab2 else 3
    variant, variant_ms = model.autotune()        # tile variant of the tendency kernel

    model.time_step(dt, args.warmup)              # warm-up (graph capture, clocks)
    model.synchronize()
    # ---- timed region: K steps, kernel events on the model stream
    model.set_option(ocn.OCN_OPT_KERNEL_TIMING, 1)
    clocks = ClockSampler(local)
    time.sleep(0.4)
    barrier(world)
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(model.stream)
    model.time_step(dt, args.steps)
    e1.record(model.stream)
    torch.cuda.synchronize(dev)
    barrier(world)
    ck = clocks.stop()
    ms_local = e0.elapsed_time(e1)
    ktimes = model.kernel_times()
    model.set_option(ocn.OCN_OPT_KERNEL_TIMING, 0)
    launches = sum(c for c, _ in ktimes.values())
    ms = max_over_ranks(ms_local, world)
    value = cells * substeps * args.steps * world / (ms * 1e-3)
    d = model.diagnostics(dt)

    # ---- e2e: through the C ABI with pinned host buffers, copies inside the timed region
    names = ["u", "v", "w"] + model.tracers
    npt, tdt = (np.float32, torch.float32) if p["precision"] == 32 else (np.float64, torch.float64)
    host_in = {n: torch.from_numpy(np.ascontiguousarray(st[n], dtype=npt)).pin_memory() for n in names}
    host_out = {n: torch.empty(model.shape(n), dtype=tdt).pin_memory() for n in names}
    h2d = sum(t.numel() * t.element_size() for t in host_in.values())
    d2h = sum(t.numel() * t.element_size() for t in host_out.values())
    k_e2e = max(2, min(args.steps, 6))
    model.set_option(ocn.OCN_OPT_GRAPHS, 1)
    # a second instance, so that one instance's host transfers overlap the other's step
    model2 = ocn.Model(p, device=dev)
    configure(model2)
    model2.set_option(ocn.OCN_OPT_TENDENCY_VARIANT, variant)
    pair = (model, model2)
    outs = (host_out, {n: torch.empty(model.shape(n), dtype=tdt).pin_memory() for n in names})

    def put(m, wait=True):
        m.set_host_many(host_in, wait)

    def take(m, out, wait=True):
        m.get_host_many(out, wait)

    for m, out in zip(pair, outs):
        for _ in range(2):                         # warm the e2e path: both buffer parities' step graphs
            put(m); m.time_step(dt, 1); take(m, out)
    barrier(world)
    t0 = time.perf_counter()                       # serial: copy in, step, copy out, one step at a time
    for _ in range(k_e2e):
        put(model); model.time_step(dt, 1); take(model, host_out)
    t_serial = max_over_ranks(time.perf_counter() - t0, world)
    barrier(world)
    t0 = time.perf_counter()                       # pipelined over the two instances, copies not waited for
    put(pair[0], False); pair[0].time_step(dt, 1)
    for i in range(1, k_e2e):
        x, y = pair[i % 2], pair[(i - 1) % 2]
        put(x, False); x.time_step(dt, 1)          # step i's copies in and launch ...
        take(y, outs[(i - 1) % 2], False)          # ... while step i-1 finishes and is copied out
    take(pair[(k_e2e - 1) % 2], outs[(k_e2e - 1) % 2], False)
    for m in pair:                                 # every copy of every step has arrived
        m.wait_transfers()
    t_e2e = max_over_ranks(time.perf_counter() - t0, world)
    e2e_value = cells * substeps * k_e2e * world / t_e2e
    e2e_serial = cells * substeps * k_e2e * world / t_serial
    del model2
    fma_peak = max(ocn.fp32_fma_peak() for _ in range(3))     # measured ALU denominator

    if rank != 0:
        return 0
    peaks = measured_peaks()
    # dominant kernel and its roofline
    per_class = {k: {"launches": c, "ms_total": t, "ms_per_launch": (t / c if c else None),
                     "share": (t / sum(x for _, x in ktimes.values()))} for k, (c, t) in ktimes.items() if c}
    dom = max(per_class, key=lambda k: per_class[k]["ms_total"])
    model_flops = tendency_flops_per_cell(p)
    exec_flops = profiled_field("tendency", p["name"], "fp32_flops_per_cell_executed")
    clock_mhz = peaks["sm_max_mhz"]
    if dom == "tendency":
        t_launch = per_class["tendency"]["ms_per_launch"] * 1e-3
        flops_cell = exec_flops if exec_flops else model_flops
        achieved = flops_cell * cells / t_launch / 1e12
        nominal = SMS * FP32_LANES * 2 * clock_mhz * 1e6 / 1e12
        peak = fma_peak
        traffic = profiled_traffic("tendency", p["name"])
        # the HBM view of the same launch: 2 of 3 substages read G^{m-1}
        tb = (tendency_bytes_per_cell(p, True) + 2 * tendency_bytes_per_cell(p)) / 3.0
        roof = {"bound": "alu", "kernel": "k_tendency", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic,
                "traffic_source": "profiles/tendency_les_512.txt: an RK3 first-substage launch (no G_prev read), "
                                  "scaled from 256x256x128 by the cell count",
                "algorithmic": (f"{flops_cell:.0f} FP32 flops per cell executed (ncu FFMA x 2 + FMUL + FADD per cell, "
                                "profiles/tendency_les_512.txt)" if exec_flops else
                                f"{flops_cell} FP32 flops per cell from the WENO cost model (the ncu instruction count "
                                "is stale for these sources)") + f" x {cells} cells per launch",
                "cost_model_flops_per_cell": model_flops,
                "executed_flops_per_cell": exec_flops,
                "peak_source": "measured FP32 FMA throughput (ocn_fp32_fma_peak, this run)",
                "nominal_peak": nominal, "frac_of_nominal": achieved / nominal,
                "nominal_source": f"{SMS} SMs x {FP32_LANES} FP32 lanes x 2 x {clock_mhz:.0f} MHz",
                "hbm_view": {"achieved": tb * cells / t_launch / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                             "frac": tb * cells / t_launch / 1e9 / peaks["hbm_gbs"],
                             "algorithmic": f"{tb:.1f} B per cell (state in/out, G out, G_prev in on 2 of 3 "
                                            "substages, nu_e)"}}
    else:
        roof = None
    sub_bytes = substep_bytes_per_cell(p) * cells
    t_sub = ms / args.steps / substeps * 1e-3
    metric, unit = ("cell-QAB2-steps/sec", "cell-steps/s") if qab2 else ("cell-RK3-substeps/sec", "cell-substeps/s")
    vroof = None
    if "vertical" in per_class:
        nfield = 3 + len(model.tracers)
        vbytes = cells * nfield * 2 * (4 if p["precision"] == 32 else 8)
        vt = per_class["vertical"]["ms_per_launch"] * 1e-3
        # the implicit step is two kernels (the column-independent coefficients, then the segmented
        # solve), timed together as one
        kname = "k_vdiff_factor + k_vdiff_isolve" if args.vertical == "implicit" else "k_vdiff_explicit"
        vroof = {"bound": "hbm", "kernel": kname, "achieved": vbytes / vt / 1e9,
                 "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": vbytes / vt / 1e9 / peaks["hbm_gbs"],
                 "algorithmic": f"{nfield} fields x (read + write) x {4 if p['precision'] == 32 else 8} B per cell",
                 "ms_per_launch": vt * 1e3}
    line = {
        "metric": metric, "value": value, "unit": unit, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if p["precision"] == 32 else "f64",
        "data": "synthetic",
        "config": {"workload": workload_desc(p) + ("" if not qab2 else ", QAB2 (chi 0.1)") +
                               ("" if args.vertical == "none" else f", {args.vertical} vertical diffusion profile"),
                   "parallelism": "replicas" if world > 1 else "single",
                   "l2": "inputs larger than L2 (model state 1.3 GB)", "graphs": False,
                   "kernel_events": True, "tendency_variant": variant,
                   "autotune_ms": [round(x, 3) for x in variant_ms]},
        "roofline": roof,
        "substep_hbm": {"achieved": sub_bytes / t_sub / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                        "frac": sub_bytes / t_sub / 1e9 / peaks["hbm_gbs"], "peak_source": peaks["source"],
                        "algorithmic": f"{substep_bytes_per_cell(p)} B per cell per substage"},
        "kernels": per_class,
        "vertical_roofline": vroof,
        "gpu_launches": launches,
        "e2e": {"value": e2e_value, "unit": "cell-substeps/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "steps": k_e2e, "path": "ocn_set_fields/ocn_time_step/ocn_get_fields with pinned host buffers (OCN_HOST_ASYNC, "
                                        "ocn_wait_transfers before the clock stops); two model instances alternate, "
                                        "so step i's copy-in and launch precede the copy-out of step i-1",
                "serial": {"value": e2e_serial, "path": "copy in, step, copy out, one step at a time"}},
        "clocks": ck,
        "checks": {"max_div": d["max_div"], "cfl": d["cfl"], "nonfinite": d["nonfinite"]},
    }
    if args.size:
        line["config"]["workload"] += " (resized for profiling, not a bench line)"
    if world == 1 and not args.no_cpu_baseline and not qab2 and args.vertical == "none":
        kept = {}
        rate, sps, cores, sample = oracle_rate(args.workload, 1, keep=kept)
        r1, _, _, sample1 = oracle_rate(args.workload, 1, cores=1, sample=CPU_SAMPLE_1CORE)
        line["cpu_baseline"] = {"value": rate, "unit": "cell-substeps/s", "cores": cores, "kind": "oracle",
                                "sample": sample,
                                "single_core": {"value": r1, "unit": "cell-substeps/s", "cores": 1, "sample": sample1}}
        # the same sample stepped by the library, against the oracle's result (relative L2 per field)
        ps, om = kept["params"], kept["model"]
        gm = ocn.Model(ps, device=dev)
        gm.set(**inputs.initial_state(ps))
        gm.time_step(ps["dt"], kept["steps"])
        err = {}
        for n in ["u", "v", "w"] + gm.tracers:
            ref = om.get(n)
            err[n] = float(np.linalg.norm(gm.get_numpy(n).astype(np.float64) - ref) / max(np.linalg.norm(ref), 1e-300))
        line["oracle_error"] = {"rel_l2": err, "sample": sample, "precision": f"FP{ps['precision']} vs the FP64 oracle"}
        del gm
    print(json.dumps(line), flush=True)
    return 0


def run_ensemble(args, world, rank, local):
    """Ensemble of uneven members: one graph per step in which every kernel is one batched launch
    over all members (the headline), against the same graph with a branch of per-member launches
    per member (concurrent) and against members stepped one after the other, on the same GPU."""
    import torch
    from paper_2502_14148_gb300 import build, inputs, ocn
    if rank == 0 or world == 1:
        build.build()
    barrier(world)
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    if args.ensemble_mode is None:
        args.ensemble_mode = "concurrent"
    ps = inputs.ensemble_configs(n=args.members)
    cells = sum(p["Nx"] * p["Ny"] * p["Nz"] for p in ps)
    E = ocn.Ensemble(ps, device=dev)
    for i, p in enumerate(ps):
        E.members[i].set(**inputs.initial_state(p, seed=inputs.SEED + i + 1000 * rank))
    variants = E.autotune()
    dt = ps[0]["dt"]
    timings = {}
    launches = {}
    for mode in (args.ensemble_mode,) + tuple(m for m in ("batched", "concurrent", "sequential") if m != args.ensemble_mode):
        E.set_mode(mode)
        E.time_step(dt, args.warmup)
        E.synchronize()
        launches[mode] = E.launches_per_step()
        ck = ClockSampler(local) if mode == args.ensemble_mode else None
        barrier(world)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(E.stream)
        E.time_step(dt, args.steps)
        e1.record(E.stream)
        torch.cuda.synchronize(dev)
        barrier(world)
        timings[mode] = (max_over_ranks(e0.elapsed_time(e1), world), ck.stop() if ck else None)
    if rank != 0:
        return 0
    ms_c, clocks = timings[args.ensemble_mode]
    ms_s, _ = timings["sequential"]
    val = cells * 3 * args.steps * world / (ms_c * 1e-3)
    mode_text = {"batched": "one CUDA graph per step; every kernel one launch over all members (work list of "
                            "(member, block))",
                 "concurrent": "one CUDA graph per step, a branch of per-member launches per member",
                 "sequential": "members stepped one after the other (each with its own graph)"}
    others = {m: {"value": cells * 3 * args.steps * world / (timings[m][0] * 1e-3),
                  "ms_per_step": timings[m][0] / args.steps, "launches_per_step": launches[m], "mode": mode_text[m]}
              for m in timings if m != args.ensemble_mode}
    d = E.members[0].diagnostics(dt)
    line = {"metric": "cell-RK3-substeps/sec", "value": val, "unit": "cell-substeps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_c / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"ensemble of {len(ps)} CBL LES members ({cells/1e6:.1f} M cells; Nx=Ny in "
                                   f"{{64,96,128}}, Nz in {{64,80,96}}, WENO5, AMD, FP32, dt={dt} s)",
                       "mode": mode_text[args.ensemble_mode],
                       "tendency_variants": sorted(set(variants))},
            "gpu_launches": launches[args.ensemble_mode] * args.steps,
            "other_modes": others,
            "speedup_vs_sequential": ms_s / ms_c, "clocks": clocks,
            "checks": {"member0_max_div": d["max_div"], "member0_nonfinite": d["nonfinite"]}}
    print(json.dumps(line), flush=True)
    return 0


def run_closure(args, world, rank, local):
    """Coarse runs with the learned column closure: args.members coarse CBL instances of 16 x 16
    columns (each on its forcing's vertical grid), AMD + the trained closure against plain AMD,
    both one graph per ensemble step.  The closure is first trained by the library (a 32-forcing,
    3 h experiment whose held-out errors are reported); the fused tensor-core closure kernel is
    then timed alone on the same number of faces for its roofline."""
    import torch
    from paper_2502_14148_gb300 import build, closure, inputs, ocn
    if rank == 0 or world == 1:
        build.build()
    barrier(world)
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    if args.ensemble_mode is None:
        args.ensemble_mode = "batched"
    t0 = time.time()
    res = closure.experiment(n_members=32, n_train=24, t_end=3 * 3600.0, dt=10.0, every=180, train_steps=2000,
                             log=lambda *a: None,
                             variants={"mlp": closure.DEFAULT_VARIANT, "cfg5": closure.DIFFUSIVITY_VARIANT})
    t_exp = time.time() - t0
    cls = {}
    for v in ("mlp", "cfg5"):
        net, mu, sigma, scale, ysc, form = res["nets"][v]
        cls[v] = closure.closure_for(net, mu, sigma, scale, ysc, form)

    def attach(model, p, v="mlp"):
        cl = cls[v]
        c = cl(p) if callable(cl) else cl
        model.set_column_closure(c[0], c[1], c[2], c[3], p["N2"], mode=c[4])
    fine = inputs.ensemble_configs(n=args.members, seed=inputs.SEED + 7, dt=10.0)
    ps = [closure.coarse_config(p) for p in fine]
    cells = sum(p["Nx"] * p["Ny"] * p["Nz"] for p in ps)
    faces = sum(p["Nx"] * p["Ny"] * (p["Nz"] + 1) for p in ps)
    dt = 10.0
    timings = {}
    for mode in ("plain", "learned", "cfg5"):
        E = ocn.Ensemble(ps, device=dev)
        E.set_mode(args.ensemble_mode)
        for i, p in enumerate(ps):
            E.members[i].set(**inputs.initial_state(p, seed=inputs.SEED + i + 1000 * rank))
            if mode != "plain":
                attach(E.members[i], p, "mlp" if mode == "learned" else "cfg5")
        E.autotune()
        E.time_step(dt, args.warmup)
        E.synchronize()
        ck = ClockSampler(local) if mode == "learned" else None
        barrier(world)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(E.stream)
        E.time_step(dt, args.steps)
        e1.record(E.stream)
        torch.cuda.synchronize(dev)
        barrier(world)
        d = E.members[0].diagnostics(dt)
        timings[mode] = (max_over_ranks(e0.elapsed_time(e1), world), ck.stop() if ck else None, E.launches_per_step(), d)
        del E
    # the fused closure kernel alone, on one model with as many faces (same kernel, one launch)
    side = 256
    nz = max(8, int(round(faces / (side * side))) - 1)
    q = closure.coarse_config(dict(fine[0], Nz=nz, z_faces=inputs.tanh_faces(nz, fine[0]["Lz"])), side, side)
    big = ocn.Model(q, device=dev)
    big.set(**inputs.initial_state(q, seed=inputs.SEED))
    attach(big, q)
    nsamp = side * side * (nz + 1)
    F = torch.empty((3, nz + 1, side, side), dtype=torch.float32, device=dev)
    reps = 20
    for _ in range(3):
        big.column_fluxes(learned=True)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(big.stream):
        e0.record(big.stream)
        for _ in range(reps):
            ocn.lib().ocn_column_fluxes(big._h, 1, ocn.C.c_void_p(F.data_ptr()))
        e1.record(big.stream)
    torch.cuda.synchronize(dev)
    t_kernel = e0.elapsed_time(e1) / reps * 1e-3
    if rank != 0:
        return 0
    peaks = measured_peaks()
    ms_p, _, _, _ = timings["plain"]
    ms_l, clocks, launches, d = timings["learned"]
    ms_5, _, launches5, _ = timings["cfg5"]
    val = cells * 3 * args.steps * world / (ms_l * 1e-3)
    achieved = MLP_FLOPS_PER_SAMPLE * nsamp / t_kernel / 1e12
    s = res["summary"]
    line = {"metric": "cell-RK3-substeps/sec", "value": val, "unit": "cell-substeps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_l / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 state, bf16 network", "data": "synthetic",
            "config": {"workload": f"{len(ps)} coarse CBL instances of 16x16 columns ({cells/1e6:.2f} M cells, "
                                   f"{faces/1e6:.2f} M closure faces per substage; Nz in {{64,80,96}}, WENO5, "
                                   f"AMD + learned column closure, FP32, dt={dt} s)",
                       "mode": {"batched": "one CUDA graph per ensemble step; every kernel one launch over all "
                                            "members", "concurrent": "one CUDA graph per ensemble step, members on "
                                            "concurrent branches", "sequential": "members one after the other"}[
                                                args.ensemble_mode]},
            "gpu_launches": launches * args.steps,
            "plain_amd": {"value": cells * 3 * args.steps * world / (ms_p * 1e-3), "ms_per_step": ms_p / args.steps},
            "closure_overhead": ms_l / ms_p,
            "cfg5_closure": {"value": cells * 3 * args.steps * world / (ms_5 * 1e-3), "ms_per_step": ms_5 / args.steps,
                             "launches_per_step": launches5,
                             "closure": "network on the local gradients (5 faces) + surface buoyancy flux + f, "
                                        "diffusivities applied by the implicit vertical solve"},
            "roofline": {"bound": "tensor", "kernel": "k_mlp_closure", "achieved": achieved,
                         "peak": peaks["bf16_tflops"], "unit": "TFLOP/s", "frac": achieved / peaks["bf16_tflops"],
                         "traffic": None,
                         "algorithmic": f"{MLP_FLOPS_PER_SAMPLE} flops per face x {nsamp} faces per launch",
                         "peak_source": f"{peaks['source']} bf16 burst", "ms_per_launch": t_kernel * 1e3},
            "flux_error": {"held_out_forcings": s["n_members"] - s["n_train"],
                           "b_profile": {"plain_amd": s["amd_b"], "learned": s["mlp_b"], "cfg5": s["cfg5_b"]},
                           "buoyancy_flux": {"plain_amd": s["amd_Fb"], "learned": s["mlp_Fb"], "cfg5": s["cfg5_Fb"]},
                           "training_samples": s["mlp_samples"], "experiment_seconds": t_exp,
                           "definition": "normalised RMS vs coarse-grained fine LES over 30-min snapshots to 3 h"},
            "clocks": clocks,
            "checks": {"member0_max_div": d["max_div"], "member0_nonfinite": d["nonfinite"]}}
    print(json.dumps(line), flush=True)
    return 0


def run_closure_kernel(args, world, rank, local):
    """The fused tensor-core closure kernel alone (features -> 4-layer BF16 network -> fluxes) on
    one FP32 CBL model of --size (default 256x256x80 = 5.3 M faces, the face count of 256 coarse
    16 x 16 instances), with the seeded initial network: its cost does not depend on training."""
    import torch
    from paper_2502_14148_gb300 import build, closure, inputs, ocn
    if rank == 0 or world == 1:
        build.build()
    barrier(world)
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    nx, ny, nz = (int(x) for x in (args.size or "256x256x80").split("x"))
    base = inputs.ensemble_configs(n=1, dt=10.0)[0]
    q = closure.coarse_config(dict(base, Nz=nz, z_faces=inputs.tanh_faces(nz, base["Lz"])), nx, ny)
    m = ocn.Model(q, device=dev)
    m.set(**inputs.initial_state(q, seed=inputs.SEED + rank))
    net = ocn.MLP(inputs.MLP_SIZES, max_batch=1024, device=dev)
    net.set_params(inputs.mlp_init())
    X = m.closure_features(q["N2"])
    mu, sigma = closure.normalisation(X)
    m.set_column_closure(net, mu, sigma, (q["top_flux"]["b"], 0.0, 0.0), q["N2"])
    nsamp = nx * ny * (nz + 1)
    F = torch.empty((3, nz + 1, ny, nx), dtype=torch.float32, device=dev)
    for _ in range(max(args.warmup, 1)):
        ocn._check(ocn.lib().ocn_column_fluxes(m._h, 1, ocn.C.c_void_p(F.data_ptr())), "ocn_column_fluxes")
    torch.cuda.synchronize(dev)
    ck = ClockSampler(local)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(m.stream)
    for _ in range(args.steps):
        ocn._check(ocn.lib().ocn_column_fluxes(m._h, 1, ocn.C.c_void_p(F.data_ptr())), "ocn_column_fluxes")
    e1.record(m.stream)
    torch.cuda.synchronize(dev)
    clocks = ck.stop()
    t = max_over_ranks(e0.elapsed_time(e1) / args.steps, world) * 1e-3
    if rank != 0:
        return 0
    peaks = measured_peaks()
    achieved = MLP_FLOPS_PER_SAMPLE * nsamp / t / 1e12
    line = {"metric": "closure faces/sec", "value": nsamp * world / t, "unit": "faces/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16 (fp32 accumulate)", "data": "synthetic",
            "config": {"workload": f"learned column closure kernel, {nx}x{ny}x{nz} FP32 CBL state, {nsamp} faces",
                       "launches_per_step": 2},
            "roofline": {"bound": "tensor", "kernel": "k_mlp_closure", "achieved": achieved, "peak": peaks["bf16_tflops"],
                         "unit": "TFLOP/s", "frac": achieved / peaks["bf16_tflops"],
                         "traffic": profiled_traffic("mlp_closure", f"{nx}x{ny}x{nz}"),
                         "algorithmic": f"{MLP_FLOPS_PER_SAMPLE} flops per face x {nsamp} faces per launch",
                         "peak_source": f"{peaks['source']} bf16 burst"},
            "gpu_launches": 2 * args.steps, "clocks": clocks}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="les_512", help="les_512 (default), cbl_256, taylor_green_32, ensemble, closure or closure_kernel")
    ap.add_argument("--members", type=int, default=None,
                    help="instances: ensemble members (--workload ensemble, default 64) or coarse instances "
                         "(--workload closure, default 256)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ensemble-mode", default=None, choices=["batched", "concurrent", "sequential"],
                    help="how the ensemble and closure workloads step their members (default: concurrent for "
                         "the ensemble of fine members, batched for the coarse instances of the closure workload)")
    ap.add_argument("--stepper", default="rk3", choices=["rk3", "qab2"], help="time stepper (default RK3)")
    ap.add_argument("--vertical", default="none", choices=["none", "explicit", "implicit"],
                    help="add a vertical diffusivity profile, explicit or semi-implicit")
    ap.add_argument("--size", default=None, help="NxxNyxNz: the workload's physics and spacing on another grid (profiling)")
    args = ap.parse_args()
    world, rank, local = dist_setup()
    try:
        if args.impl == "reference":
            return run_reference(args, world, rank)
        if args.workload == "ensemble":
            args.members = args.members or 64
            return run_ensemble(args, world, rank, local)
        if args.workload == "closure":
            args.members = args.members or 256
            return run_closure(args, world, rank, local)
        if args.workload == "closure_kernel":
            return run_closure_kernel(args, world, rank, local)
        return run_ours(args, world, rank, local)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
