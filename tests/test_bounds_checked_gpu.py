"""The bounds-checked build (a test aid in place of a memory checker): every translation unit
compiled with -DOCN_BOUNDS_CHECK=1 into libocn_checked.so, whose tendency kernel, projection FFTs
and tridiagonal solve record an out-of-range index in the model's status word instead of
accessing it.  A subprocess loads that variant (OCN_LIBRARY) and runs the tiny and ragged cases
of the parity suite -- one to five levels, fewer levels than the stencils and the staging depth,
4x4 tiles that wrap the periodic domain, ragged multi-tile grids, stretched z, both WENO orders,
Smagorinsky-Lilly and AMD, FP64 and FP32 -- through a tendency evaluation (against the FP64
oracle at the suite's bars), a projection, two RK3 steps and a batched ensemble step; every
model's status word must stay 0."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r'''
import sys
import numpy as np
sys.path.insert(0, sys.argv[1])
from paper_2502_14148_gb300 import inputs, ocn
from oracle import oracle

def params(**over):
    p = dict(Nx=36, Ny=18, Nz=12, Lx=36.0, Ly=18.0, Lz=12.0, stretch=1.5, precision=64, weno_order=5,
             closure="none", nu=0.02, kappa=0.01, Cs=0.16, Cb=1.0, Pr=0.7, C_amd=1 / 12, f=0.3,
             tracers=["b"], eos="buoyancy_tracer")
    p.update(over)
    p["z_faces"] = inputs.tanh_faces(p["Nz"], p["Lz"], p["stretch"]) if p.get("stretch") else inputs.uniform_faces(p["Nz"], p["Lz"])
    p.setdefault("top_flux", {})
    p.setdefault("bottom_flux", {})
    return p

def rounded(st, precision):
    return {k: v.astype(np.float32).astype(np.float64) for k, v in st.items()} if precision == 32 else st

def rel_max(a, o):
    a = np.asarray(a, dtype=np.float64); o = np.asarray(o, dtype=np.float64)
    return np.abs(a - o).max() / max(np.abs(o).max(), 1e-300)

ncase = 0
for precision in (64, 32):
    for dims in [(4, 4, 1), (4, 4, 2), (6, 4, 3), (12, 8, 5), (72, 36, 24)]:
        for order in (5, 9):
            for closure in ("smagorinsky", "amd"):
                Nx, Ny, Nz = dims
                p = params(Nx=Nx, Ny=Ny, Nz=Nz, Lx=float(Nx), Ly=float(Ny), Lz=float(Nz), precision=precision,
                           weno_order=order, closure=closure, tracers=["T", "S"], eos="linear_ts",
                           top_flux={"u": 1e-2, "T": 2e-3})
                st = rounded(inputs.random_state(p, seed=41, amp=0.7), precision)
                st["T"] = 20.0 + 0.5 * st["T"]
                st["S"] = 35.0 + 0.1 * st["S"]
                st = rounded(st, precision)
                g = ocn.Model(p)
                g.set(project=False, **st)
                G = {k: v.cpu().numpy() for k, v in g.compute_tendencies().items()}
                o = oracle.OracleModel(p)
                o.set(**st)
                O = o.tendencies()
                tol = 1e-11 if precision == 64 else 2e-5
                for name in O:
                    err = rel_max(G[name], O[name])
                    assert err < tol, (dims, order, closure, precision, name, err)
                g.project()
                g.time_step(0.05, 2)
                status, checked = g.bounds_status()
                assert checked, "the loaded library is not the bounds-checked variant"
                assert status == 0, (dims, order, closure, precision, hex(status))
                ncase += 1
ps = inputs.ensemble_configs(n=3, sizes=(16, 24), depths=(8, 12))
E = ocn.Ensemble(ps, device="cuda:0")
E.set_mode("batched")
for i, pm in enumerate(ps):
    E.members[i].set(**inputs.initial_state(pm, seed=inputs.SEED + i))
E.time_step(ps[0]["dt"], 1)
for m in E.members:
    status, checked = m.bounds_status()
    assert checked and status == 0, hex(status)
print("bounds-checked cases:", ncase, "+ a batched ensemble of", len(ps))
'''


def test_tiny_and_ragged_cases_stay_in_bounds():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_14148_gb300 import build
    path = build.build(checked=True)
    env = dict(os.environ, OCN_LIBRARY=path)
    r = subprocess.run([sys.executable, "-c", SCRIPT, ROOT], env=env, capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "bounds-checked cases: 40" in r.stdout, r.stdout
