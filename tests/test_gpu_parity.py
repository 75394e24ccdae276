"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Inputs always come from the seeded generators in paper_2502_14148_gb300.inputs;
no oracle input or expected value comes from the GPU.  Tolerances:
  FP64            max|a-o| / max|o| <= 1e-11 per field
  FP32 runs       ||a-o||_2 / ||o||_2 <= 1e-4 per field after 100 steps
  FP32 one call   max|a-o| / max|o| <= 2e-5 (inputs rounded to FP32 on both sides)
"""
import math

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


def rel_max(a, o):
    a = np.asarray(a, dtype=np.float64); o = np.asarray(o, dtype=np.float64)
    return np.abs(a - o).max() / max(np.abs(o).max(), 1e-300)


def rel_l2(a, o):
    a = np.asarray(a, dtype=np.float64); o = np.asarray(o, dtype=np.float64)
    return np.linalg.norm(a - o) / max(np.linalg.norm(o), 1e-300)


def params(**over):
    p = dict(Nx=36, Ny=18, Nz=12, Lx=36.0, Ly=18.0, Lz=12.0, stretch=1.5, precision=64, weno_order=5,
             closure="none", nu=0.02, kappa=0.01, Cs=0.16, Cb=1.0, Pr=0.7, C_amd=1 / 12, f=0.3,
             tracers=["b"], eos="buoyancy_tracer")
    p.update(over)
    if p.get("stretch"):
        p["z_faces"] = inputs.tanh_faces(p["Nz"], p["Lz"], p["stretch"])
    else:
        p["z_faces"] = inputs.uniform_faces(p["Nz"], p["Lz"])
    p.setdefault("top_flux", {})
    p.setdefault("bottom_flux", {})
    return p


def rounded(st, precision):
    if precision == 32:
        return {k: v.astype(np.float32).astype(np.float64) for k, v in st.items()}
    return st


# ----------------------------------------------------------------------------- projection
@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("dims", [(36, 24, 10), (48, 18, 7), (16, 16, 16), (4, 6, 1), (96, 8, 3)])
def test_projection_parity(ocn, oracle_mod, precision, dims):
    Nx, Ny, Nz = dims
    p = params(Nx=Nx, Ny=Ny, Nz=Nz, Lx=float(Nx), Ly=float(Ny) * 0.7, Lz=float(Nz), precision=precision)
    st = rounded(inputs.random_state(p, seed=31), precision)
    g = ocn.Model(p)
    g.set(project=False, **st)
    g.project()
    o = oracle_mod.OracleModel(p)
    o.set(**st)
    o.project(1.0)
    tol = 1e-11 if precision == 64 else 2e-5
    for name in ("u", "v", "w", "p"):
        assert rel_max(g.get_numpy(name), o.get(name)) < tol, name
    d = g.diagnostics()
    umax = max(np.abs(st[x]).max() for x in "uvw")
    assert d["max_div"] < (1e-12 if precision == 64 else 3e-5) * umax


# ----------------------------------------------------------------------------- tendencies
CASES = [
    dict(weno_order=5, closure="none"),
    dict(weno_order=5, closure="scalar"),
    dict(weno_order=5, closure="amd"),
    dict(weno_order=5, closure="smagorinsky", tracers=["T", "S"], eos="linear_ts"),
    dict(weno_order=9, closure="smagorinsky", tracers=["T", "S"], eos="linear_ts",
         top_flux={"u": -1e-2, "T": 5e-3}, bottom_flux={"v": 2e-3}),
    dict(weno_order=9, closure="amd", top_flux={"b": 1e-2}),
    dict(weno_order=9, closure="scalar", tracers=["b", "c"], stretch=None),
    dict(weno_order=5, closure="amd", tracers=["b", "c"], top_flux={"c": -3e-3}),
]


def _tendency_pair(ocn, oracle_mod, case, precision, seed=41, **over):
    p = params(precision=precision, **dict(case, **over))
    st = rounded(inputs.random_state(p, seed=seed, amp=0.7), precision)
    if p["eos"] == "linear_ts":
        st["T"] = 20.0 + 0.5 * st["T"]
        st["S"] = 35.0 + 0.1 * st["S"]
        st = rounded(st, precision)
    g = ocn.Model(p)
    g.set(project=False, **st)
    G = {k: v.cpu().numpy() for k, v in g.compute_tendencies().items()}
    o = oracle_mod.OracleModel(p)
    o.set(**st)
    return G, o.tendencies(), p


@pytest.mark.parametrize("case", CASES, ids=[f"weno{c['weno_order']}-{c['closure']}-{len(c.get('tracers', ['b']))}tr" for c in CASES])
def test_tendency_parity_fp64(ocn, oracle_mod, case):
    G, O, p = _tendency_pair(ocn, oracle_mod, case, 64)
    for name in O:
        assert rel_max(G[name], O[name]) < 1e-11, name


@pytest.mark.parametrize("case", CASES, ids=[f"weno{c['weno_order']}-{c['closure']}-{len(c.get('tracers', ['b']))}tr" for c in CASES])
def test_tendency_parity_fp32(ocn, oracle_mod, case):
    G, O, p = _tendency_pair(ocn, oracle_mod, case, 32)
    for name in O:
        assert rel_max(G[name], O[name]) < 2e-5, name


@pytest.mark.parametrize("dims", [(4, 4, 1), (4, 4, 2), (6, 4, 3), (12, 8, 5), (72, 36, 24)])
def test_tendency_parity_edge_sizes(ocn, oracle_mod, dims):
    """Degenerate and ragged sizes: a single level, fewer levels than the stencil, tiles that
    wrap the periodic domain several times, and several tiles with ragged tails."""
    Nx, Ny, Nz = dims
    for order in (5, 9):
        case = dict(weno_order=order, closure="smagorinsky", tracers=["T", "S"], eos="linear_ts",
                    top_flux={"u": 1e-2, "T": 2e-3})
        G, O, _ = _tendency_pair(ocn, oracle_mod, case, 64, Nx=Nx, Ny=Ny, Nz=Nz, Lx=float(Nx), Ly=float(Ny), Lz=float(Nz))
        for name in O:
            assert rel_max(G[name], O[name]) < 1e-11, (order, name)


@pytest.mark.parametrize("dims", [(4, 4, 1), (4, 4, 2), (6, 4, 3), (12, 8, 5), (72, 36, 24)])
@pytest.mark.parametrize("order", [5, 9])
@pytest.mark.parametrize("closure", ["smagorinsky", "amd"])
def test_tendency_parity_fp32_fused_closure_edge_sizes(ocn, oracle_mod, dims, order, closure):
    """The FP32 Smagorinsky-Lilly and AMD kernels compute the eddy diffusivities in their own z march
    (two levels ahead of the fluxes, from planes staged four levels ahead): one to five levels, fewer
    levels than the staging depth, tiles that wrap the periodic domain, ragged multi-tile grids."""
    Nx, Ny, Nz = dims
    case = dict(weno_order=order, closure=closure, tracers=["T", "S"], eos="linear_ts",
                top_flux={"u": 1e-2, "T": 2e-3})
    G, O, _ = _tendency_pair(ocn, oracle_mod, case, 32, Nx=Nx, Ny=Ny, Nz=Nz, Lx=float(Nx), Ly=float(Ny), Lz=float(Nz))
    for name in O:
        assert rel_max(G[name], O[name]) < 2e-5, (order, name)


@pytest.mark.parametrize("precision", [32, 64])
@pytest.mark.parametrize("eos", ["linear_ts", "buoyancy_tracer"])
@pytest.mark.parametrize("closure", ["smagorinsky", "amd"])
def test_eddy_viscosity_field_matches_oracle(ocn, oracle_mod, precision, eos, closure):
    """nu_e left in the arena by a tendency evaluation (computed inside the FP32 tendency kernel,
    by the closure kernel in FP64) against the oracle's diffusivity at every cell of a stratified,
    stretched, ragged grid."""
    tracers = ["T", "S"] if eos == "linear_ts" else ["b"]
    p = params(Nx=24, Ny=18, Nz=9, precision=precision, closure=closure, tracers=tracers, eos=eos, Cb=1.0,
               Pr=0.7)
    # velocity amplitudes that put about half of the cells past the stratification cut-off
    st = inputs.random_state(p, seed=61, amp=0.01 if eos == "linear_ts" else 0.2)
    zc = 0.5 * (p["z_faces"][1:] + p["z_faces"][:-1])
    if eos == "linear_ts":
        st["T"] = 20.0 + 0.3 * zc[:, None, None] + 0.005 * st["T"]
        st["S"] = 35.0 + 0.001 * st["S"]
    else:
        st["b"] = 0.2 * zc[:, None, None] + 0.005 * st["b"]
    st = rounded(st, precision)
    g = ocn.Model(p)
    g.set(project=False, **st)
    g.compute_tendencies()
    nu = g.get_numpy("nu_e").astype(np.float64)
    o = oracle_mod.OracleModel(p)
    o.set(**st)
    ref = np.array([[[o.diffusivity_at(0, i, j, k) for i in range(p["Nx"])] for j in range(p["Ny"])]
                    for k in range(p["Nz"])])
    assert 0.3 < (ref > 0).mean() < 0.7                       # both sides of the cut-off
    if closure == "smagorinsky":
        # nu_e^2 = (C_s Delta)^4 max(|S|^2 - C_b N^2 / Pr, 0) is linear in the rounded quantities; nu_e
        # itself has an infinite slope at the cut-off, where a rounding-level change of the argument
        # moves it by the square root of the rounding unit
        assert rel_max(nu ** 2, ref ** 2) < (1e-11 if precision == 64 else 1e-5)
    else:
        assert rel_max(nu, ref) < (1e-11 if precision == 64 else 1e-5)


# ----------------------------------------------------------------------------- time stepping
def _run_pair(ocn, oracle_mod, p, steps, seed=inputs.SEED):
    st = rounded(inputs.initial_state(p, seed=seed), p["precision"])
    g = ocn.Model(p)
    g.set(**st)                      # set! projects the velocity (both sides)
    o = oracle_mod.OracleModel(p)
    o.set(**st)
    o.project(1.0)
    g.time_step(p["dt"], steps)
    o.time_step(p["dt"], steps)
    return g, o


def test_taylor_green_32_fp64_20_steps(ocn, oracle_mod):
    """32^3, L = 2 pi, FP64, WENO5, nu = 1e-3, b = 0.01 z, Taylor-Green + N(0,1e-3) noise,
    dt = 1e-2, 20 RK3 steps: every field within 1e-11 of the oracle; divergence at round-off;
    tracer and horizontal momentum conserved."""
    p = inputs.config("taylor_green_32")
    g, o = _run_pair(ocn, oracle_mod, p, p["steps"])
    for name in ("u", "v", "w", "b"):
        assert rel_max(g.get_numpy(name), o.get(name)) < 1e-11, name
    dg, do = g.diagnostics(p["dt"]), o.diagnostics(p["dt"])
    assert dg["max_div"] < 1e-12
    assert abs(dg["sum_b"] - do["sum_b"]) < 1e-12 * abs(do["sum_b"])
    g0 = ocn.Model(p)
    g0.set(**inputs.initial_state(p))
    d0 = g0.diagnostics()
    assert abs(dg["sum_b"] - d0["sum_b"]) < 1e-12 * abs(d0["sum_b"])
    assert abs(dg["sum_u"] - d0["sum_u"]) < 1e-13 * 32 ** 3 * (2 * math.pi / 32) ** 3


def test_cbl_fp32_100_steps(ocn, oracle_mod):
    """Convective boundary layer physics (WENO5, AMD, f = 1e-4, surface buoyancy flux 1e-8,
    N^2 = 1e-5, tanh-stretched z, noise) at 48x48x24 with the cbl_256 spacing: FP32 fields
    after 100 steps within 1e-4 (L2, relative) of the FP64 oracle."""
    p = inputs.config("cbl_256", Nx=48, Ny=48, Nz=24)
    g, o = _run_pair(ocn, oracle_mod, p, 100)
    for name in ("u", "v", "w", "b"):
        assert rel_l2(g.get_numpy(name), o.get(name)) < 1e-4, name


def test_les_fp32_100_steps(ocn, oracle_mod):
    """Wind- and convection-driven LES physics (WENO9, Smagorinsky-Lilly, T and S with a linear
    EOS, f = 1e-4, surface stress and heat flux, noise) at 36x36x24, 1 m spacing: FP32 fields after
    100 steps within 1e-4 (L2, relative) of the FP64 oracle."""
    p = inputs.config("les_512", Nx=36, Ny=36, Nz=24)
    g, o = _run_pair(ocn, oracle_mod, p, 100)
    for name in ("u", "v", "w", "T", "S"):
        assert rel_l2(g.get_numpy(name), o.get(name)) < 1e-4, name
    # temperature anomaly relative to its own variation, not to T0
    T0 = p["T0"]
    assert rel_l2(g.get_numpy("T") - T0, o.get("T") - T0) < 1e-4


def _full_size_sampled(ocn, oracle_mod, p, names, tol):
    """Tendencies at 300 sampled points against the oracle's pointwise evaluation (the one-call
    FP32 bar: max|a-o| / max|o| over the samples), and the projection checked by properties that hold at any size (div u = 0, u_new = u - grad p,
    lap p = div u), on the workload's full grid."""
    st = rounded(inputs.initial_state(p), 32)
    g = ocn.Model(p)
    g.set(project=False, **st)
    G = {k: v.cpu().numpy() for k, v in g.compute_tendencies().items()}
    o = oracle_mod.OracleModel(p)
    o.set(**st)
    rng = np.random.default_rng(5)
    Nx, Ny, Nz = p["Nx"], p["Ny"], p["Nz"]
    pts = [(int(rng.integers(Nx)), int(rng.integers(Ny)), int(k)) for k in
           list(rng.integers(0, Nz, 240)) + [0, 1, 2, 3, 4, 5, Nz - 6, Nz - 5, Nz - 4, Nz - 3, Nz - 2, Nz - 1] * 5]
    for name in names:
        ref = np.array([o.tendency_at(name, i, j, k) for (i, j, k) in pts])
        got = np.array([G[name][k, j, i] for (i, j, k) in pts])
        scale = max(np.abs(ref).max(), 1e-30)
        print(p["name"], "sampled tendency", name, f"{np.abs(got - ref).max() / scale:.2e}")
        assert np.abs(got - ref).max() / scale < tol, name
    # projection properties
    u0, v0, w0 = (st[x] for x in "uvw")
    g.project()
    u1, v1, w1, pr = (g.get_numpy(x).astype(np.float64) for x in ("u", "v", "w", "p"))
    d = g.diagnostics()
    assert d["max_div"] < 1e-5 * np.abs(u0).max() * max(Nx / p["Lx"], 1.0)
    dx, dy = p["Lx"] / Nx, p["Ly"] / Ny
    zf = np.asarray(p["z_faces"]); zc = 0.5 * (zf[1:] + zf[:-1]); dzc = np.diff(zf)
    us = max(np.abs(u0).max(), 1e-30)
    for (i, j, k) in pts[:100]:
        assert abs(u1[k, j, i] - (u0[k, j, i] - (pr[k, j, i] - pr[k, j, i - 1]) / dx)) < 1e-5 * max(us, 1.0)
        assert abs(v1[k, j, i] - (v0[k, j, i] - (pr[k, j, i] - pr[k, j - 1, i]) / dy)) < 1e-5 * max(us, 1.0)
        if 0 < k < Nz:
            assert abs(w1[k, j, i] - (w0[k, j, i] - (pr[k, j, i] - pr[k - 1, j, i]) / (zc[k] - zc[k - 1]))) < 1e-5 * max(us, 1.0)
        ip, jp = (i + 1) % Nx, (j + 1) % Ny
        div0 = (u0[k, j, ip] - u0[k, j, i]) / dx + (v0[k, jp, i] - v0[k, j, i]) / dy + (w0[k + 1, j, i] - w0[k, j, i]) / dzc[k]
        lap = (pr[k, j, ip] - 2 * pr[k, j, i] + pr[k, j, i - 1]) / dx ** 2 + (pr[k, jp, i] - 2 * pr[k, j, i] + pr[k, j - 1, i]) / dy ** 2
        up = (pr[k + 1, j, i] - pr[k, j, i]) / (zc[k + 1] - zc[k]) if k + 1 < Nz else 0.0
        dn = (pr[k, j, i] - pr[k - 1, j, i]) / (zc[k] - zc[k - 1]) if k > 0 else 0.0
        lap += (up - dn) / dzc[k]
        assert abs(lap - div0) < 1e-4 * max(1.0, abs(div0)), (i, j, k)


def test_les_512_full_size_sampled(ocn, oracle_mod):
    """The benchmark workload at full size (512x512x256 FP32, WENO9, Smagorinsky-Lilly, T,S)."""
    _full_size_sampled(ocn, oracle_mod, inputs.config("les_512"), ("u", "v", "w", "T", "S"), 2e-5)


def test_cbl_256_full_size_sampled(ocn, oracle_mod):
    """The convective-boundary-layer configuration at full size (256x256x128 FP32, 2 m spacing,
    tanh-stretched z, WENO5, AMD, f = 1e-4, surface buoyancy flux)."""
    _full_size_sampled(ocn, oracle_mod, inputs.config("cbl_256"), ("u", "v", "w", "b"), 2e-5)


# ----------------------------------------------------------------------------- behaviour
def test_graph_replay_matches_direct_launches(ocn):
    p = inputs.config("les_512", Nx=64, Ny=48, Nz=16)
    st = inputs.initial_state(p)
    a = ocn.Model(p); a.set(**st)
    b = ocn.Model(p); b.set(**st); b.set_option(ocn.OCN_OPT_GRAPHS, 0)
    a.time_step(p["dt"], 4)
    b.time_step(p["dt"], 4)
    for name in ("u", "v", "w", "T", "S"):
        assert np.array_equal(a.get_numpy(name), b.get_numpy(name)), name
    assert a.launches_per_step() == b.launches_per_step() > 0


@pytest.mark.parametrize("workload", ["les_512", "cbl_256"])
def test_tendency_variants_identical(ocn, workload):
    """Every tile variant of the FP32 kernel computes exactly the same tendencies and steps
    (only the assignment of faces to threads changes), on a grid with ragged tiles, for both
    kernel families (WENO9 + Smagorinsky + T,S and WENO5 + AMD + b)."""
    p = inputs.config(workload, Nx=72, Ny=54, Nz=20)
    st = inputs.initial_state(p)
    rnd = inputs.random_state(p, seed=5, amp=0.02)
    for k in ("u", "v", "w"):
        st[k] = st[k] + rnd[k]
    ref = None
    for v in range(ocn.TENDENCY_VARIANTS):
        m = ocn.Model(p)
        m.set(**st)
        m.set_option(ocn.OCN_OPT_TENDENCY_VARIANT, v)
        G = {k: x.cpu().numpy() for k, x in m.compute_tendencies().items()}
        m.time_step(p["dt"], 2)
        out = {n: m.get_numpy(n) for n in ["u", "v", "w"] + list(p["tracers"])}
        if ref is None:
            ref = (G, out)
            continue
        for k in G:
            assert np.array_equal(G[k], ref[0][k]), (v, k)
        for k in out:
            assert np.array_equal(out[k], ref[1][k]), (v, k)
    best, ms = m.autotune()
    assert 0 <= best < ocn.TENDENCY_VARIANTS and all(x > 0 for x in ms)


def test_checkpoint_resume_bitwise(ocn):
    """A run split at a step boundary and resumed from the saved state equals the continuous run."""
    p = inputs.config("cbl_256", Nx=64, Ny=32, Nz=16)
    st = inputs.initial_state(p)
    a = ocn.Model(p); a.set(**st); a.time_step(p["dt"], 6)
    b = ocn.Model(p); b.set(**st); b.time_step(p["dt"], 3)
    saved = b.checkpoint()
    del b
    c = ocn.Model(p); c.restore(saved); c.time_step(p["dt"], 3)
    for name in ("u", "v", "w", "b"):
        assert np.array_equal(a.get_numpy(name), c.get_numpy(name)), name


def test_conservation_fp64_on_gpu(ocn):
    p = params(Nx=24, Ny=18, Nz=8, closure="amd", f=0.0, tracers=["b", "c"])
    st = inputs.random_state(p, seed=51, amp=0.3)
    g = ocn.Model(p); g.set(**st)
    d0 = g.diagnostics()
    g.time_step(0.05, 5)
    d1 = g.diagnostics()
    for key in ("sum_b", "sum_c"):
        assert abs(d1[key] - d0[key]) < 1e-13 * np.abs(st[key[4:]]).sum()
    assert abs(d1["sum_u"] - d0["sum_u"]) < 1e-13 * np.abs(st["u"]).sum()
    assert d1["max_div"] < 1e-12


def test_status_codes(ocn):
    p = params(Nx=8, Ny=8, Nz=4)
    with pytest.raises(ocn.OcnError) as ei:
        ocn.Model(dict(p, weno_order=7))
    assert ei.value.status == -7
    with pytest.raises(ocn.OcnError) as ei:
        ocn.Model(dict(p, tracers=["a", "b", "c"]))
    assert ei.value.status == -7
    with pytest.raises(ocn.OcnError) as ei:
        ocn.Model(dict(p, precision=16))
    assert ei.value.status == -1
    g = ocn.Model(p)
    st = inputs.random_state(p, seed=3)
    st["u"][1, 2, 3] = np.nan
    g.set(project=False, **st)
    d = g.diagnostics()
    assert d["status"] == "ERR_NONFINITE" and d["nonfinite"] >= 1
    g.set(project=False, u=np.full((4, 8, 8), 100.0))
    assert g.diagnostics(dt=1.0)["status"] == "ERR_CFL"
    g.time_step(0.1, 0)                 # no-op
    with pytest.raises(ocn.OcnError):
        g.time_step(float("nan"), 1)
