"""GPU parity at the sizes the measured workloads run at, and the diagnostics.

  - les_512 physics (WENO9, Smagorinsky-Lilly, T and S, linear EOS, surface stress
    and heat flux) and cbl_256 physics (WENO5, AMD, surface buoyancy flux, tanh z)
    at 128x128x64 for 100 RK3 steps in FP32 against the FP64 oracle;
  - les_512 at its full size, 512x512x256, for 3 RK3 steps (slow: the oracle
    takes about a minute per step on the host cores);
  - every diagnostic of the FP64 reductions (volume integrals, max |div u|, the
    advective CFL number, the non-finite count) against the oracle's, value by
    value, on states that are not divergence free.

Bars: FP32 fields ||a-o||_2 / ||o||_2 <= 1e-4 per field (tracers also as their
deviation from the reference value, so that T = 20 + anomaly does not hide an
error in the anomaly); FP64 1e-11 relative.  Inputs are the seeded workload
initial states; no expected value comes from the GPU.
"""
import numpy as np
import pytest

from paper_2502_14148_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ocn():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_14148_gb300 import build, ocn as mod
    build.build()
    return mod


def rel_l2(a, o):
    a = np.asarray(a, dtype=np.float64); o = np.asarray(o, dtype=np.float64)
    return np.linalg.norm(a - o) / max(np.linalg.norm(o), 1e-300)


def _rounded32(st):
    return {k: v.astype(np.float32).astype(np.float64) for k, v in st.items()}


def _run_pair(ocn, oracle_mod, p, steps):
    st = _rounded32(inputs.initial_state(p)) if p["precision"] == 32 else inputs.initial_state(p)
    g = ocn.Model(p)
    g.set(**st)                      # set! projects the velocity (both sides)
    o = oracle_mod.OracleModel(p)
    o.set(**st)
    o.project(1.0)
    g.time_step(p["dt"], steps)
    o.time_step(p["dt"], steps)
    return g, o


def _check_fields(g, o, p, tol=1e-4):
    errs = {}
    for name in ["u", "v", "w"] + list(p["tracers"]):
        a, r = g.get_numpy(name).astype(np.float64), o.get(name)
        errs[name] = rel_l2(a, r)
        if name == "T":
            errs["T-T0"] = rel_l2(a - p["T0"], r - p["T0"])
        if name == "S":
            errs["S-S0"] = rel_l2(a - p["S0"], r - p["S0"])
    print(p["name"], p["Nx"], p["Ny"], p["Nz"], {k: f"{v:.2e}" for k, v in errs.items()})
    for name, e in errs.items():
        assert e < tol, (name, e)
    return errs


def _check_diag_after_run(g, o, p):
    """After a run: integrals within FP32 storage of the oracle's, CFL within the field
    bar, and the divergence of both at their precision's round-off."""
    dg, do = g.diagnostics(p["dt"]), o.diagnostics(p["dt"])
    V = p["Lx"] * p["Ly"] * (p["z_faces"][-1] - p["z_faces"][0])
    for t in p["tracers"]:
        ref = o.get(t)
        scale = V * max(np.abs(ref).max(), 1e-30)
        assert abs(dg[f"sum_{t}"] - do[f"sum_{t}"]) < 1e-6 * scale, t
    assert abs(dg["cfl"] - do["cfl"]) < 1e-3 * do["cfl"]
    umax = max(np.abs(o.get(x)).max() for x in "uvw")
    dmin = min(p["Lx"] / p["Nx"], p["Ly"] / p["Ny"], float(np.diff(p["z_faces"]).min()))
    assert dg["max_div"] < 1e-5 * umax / dmin
    assert do["max_div"] < 1e-12 * umax / dmin
    assert dg["nonfinite"] == do["nonfinite"] == 0


def test_les_physics_128x128x64_fp32_100_steps(ocn, oracle_mod):
    """les_512 physics at 128x128x64 (1 m spacing), 100 steps of 2 s."""
    p = inputs.config("les_512", Nx=128, Ny=128, Nz=64)
    g, o = _run_pair(ocn, oracle_mod, p, 100)
    _check_fields(g, o, p)
    _check_diag_after_run(g, o, p)


def test_cbl_physics_128x128x64_fp32_100_steps(ocn, oracle_mod):
    """cbl_256 physics at 128x128x64 (2 m horizontal spacing, 256 m tanh-stretched column),
    100 steps of 10 s."""
    p = inputs.config("cbl_256", Nx=128, Ny=128, Nz=64)
    g, o = _run_pair(ocn, oracle_mod, p, 100)
    _check_fields(g, o, p)
    _check_diag_after_run(g, o, p)


@pytest.mark.slow
def test_les_512_full_size_fp32_3_steps(ocn, oracle_mod):
    """The benchmark workload itself, 512x512x256, 3 RK3 steps, every cell compared."""
    p = inputs.config("les_512")
    g, o = _run_pair(ocn, oracle_mod, p, 3)
    _check_fields(g, o, p)
    _check_diag_after_run(g, o, p)


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("closure,tracers,stretch", [("amd", ["b"], 1.5), ("smagorinsky", ["T", "S"], None)])
def test_diagnostics_match_oracle(ocn, oracle_mod, precision, closure, tracers, stretch):
    """ocn_diagnostics against the oracle's on a random, not divergence-free state (ragged,
    anisotropic, stretched or uniform z): integrals of every tracer and of u, v, w, max |div u|,
    the CFL number and the non-finite count."""
    Nx, Ny, Nz = 48, 18, 13
    p = dict(Nx=Nx, Ny=Ny, Nz=Nz, Lx=96.0, Ly=18.0, Lz=26.0, stretch=stretch, precision=precision,
             weno_order=5, closure=closure, tracers=tracers,
             eos="linear_ts" if "T" in tracers else "buoyancy_tracer", f=1e-4, top_flux={}, bottom_flux={})
    p["z_faces"] = inputs.tanh_faces(Nz, p["Lz"], stretch) if stretch else inputs.uniform_faces(Nz, p["Lz"])
    st = inputs.random_state(p, seed=71, amp=0.3)
    if "T" in tracers:
        st["T"] = 20.0 + st["T"]
        st["S"] = 35.0 + 0.1 * st["S"]
    if precision == 32:
        st = _rounded32(st)
    g = ocn.Model(p)
    g.set(project=False, **st)
    o = oracle_mod.OracleModel(p)
    o.set(**st)
    dt = 0.3
    dg, do = g.diagnostics(dt), o.diagnostics(dt)
    tol = 1e-11 if precision == 64 else 1e-6
    zf = np.asarray(p["z_faces"])
    dzc, A = np.diff(zf), p["Lx"] / Nx * p["Ly"] / Ny
    for name in tracers + ["u", "v"]:
        scale = (A * np.abs(st[name]) * dzc[:, None, None]).sum()
        assert abs(dg[f"sum_{name}"] - do[f"sum_{name}"]) < tol * scale, name
    dzf = np.diff(0.5 * (zf[1:] + zf[:-1]))
    scale_w = (A * np.abs(st["w"][1:Nz]) * dzf[:, None, None]).sum()
    assert abs(dg["sum_w"] - do["sum_w"]) < tol * scale_w
    for key in ("max_div", "cfl"):
        assert do[key] > 0.0
        assert abs(dg[key] - do[key]) < tol * do[key], (key, dg[key], do[key])
    assert dg["nonfinite"] == do["nonfinite"] == 0
