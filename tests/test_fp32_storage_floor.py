"""Why tracers are stored about a reference profile: the FP32 storage floor, measured on the oracle.

The FP64 oracle is advanced twice; in the second run the state is rounded to FP32 after every RK3 step
(arithmetic stays FP64).  With tracers rounded as they are, the mean stratification eats the FP32 digits
and w drifts by about 1e-4 in 100 CBL steps; rounding only the anomaly about the initial horizontal-mean
profile leaves a drift hundreds of times smaller.  This is a property of FP32 storage, independent of the
CUDA path.
"""
import numpy as np
import pytest

from paper_2502_14148_gb300 import inputs


def _drift(oracle_mod, p, steps, anomaly):
    st = {k: v.astype(np.float32).astype(np.float64) for k, v in inputs.initial_state(p).items()}
    ref = {t: st[t].mean(axis=(1, 2), keepdims=True) for t in p["tracers"]}
    a = oracle_mod.OracleModel(p); a.set(**st); a.project(1.0)
    b = oracle_mod.OracleModel(p); b.set(**st); b.project(1.0)
    r32 = lambda x: x.astype(np.float32).astype(np.float64)
    for _ in range(steps):
        a.time_step(p["dt"], 1)
        b.time_step(p["dt"], 1)
        upd = {f: r32(b.get(f)) for f in ("u", "v", "w")}
        for t in p["tracers"]:
            upd[t] = r32(b.get(t) - ref[t]) + ref[t] if anomaly else r32(b.get(t))
        b.set(**upd)
    wa, wb = a.get("w"), b.get("w")
    return np.linalg.norm(wa - wb) / np.linalg.norm(wa)


def test_anomaly_storage_lowers_the_fp32_floor(oracle_mod):
    p = inputs.config("cbl_256", Nx=24, Ny=24, Nz=16)
    plain = _drift(oracle_mod, p, 40, anomaly=False)
    anom = _drift(oracle_mod, p, 40, anomaly=True)
    assert plain > 20 * anom, (plain, anom)
    assert anom < 1e-5
