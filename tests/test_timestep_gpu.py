"""GPU parity of the QAB2 stepper and of vertical diffusion (explicit and semi-implicit) against
the FP64 oracle: FP64 models within 1e-11 (max relative), FP32 models within 1e-4 (relative L2)
after 100 steps."""
import numpy as np
import pytest

from paper_2502_14148_gb300 import inputs

pytestmark = pytest.mark.gpu


def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_14148_gb300 import ocn
    return torch, ocn


def _fields(p):
    return ["u", "v", "w"] + list(p.get("tracers", ["b"]))


def _compare(m, o, p, fp64, names=None):
    for n in names or _fields(p):
        a, r = m.get_numpy(n).astype(np.float64), o.get(n)
        if fp64:
            assert np.abs(a - r).max() <= 1e-11 * max(np.abs(r).max(), 1e-300), n
        else:
            assert np.linalg.norm(a - r) <= 1e-4 * np.linalg.norm(r), (n, np.linalg.norm(a - r) / np.linalg.norm(r))


def _pair(oracle_mod, ocn, p, seed=inputs.SEED):
    st = inputs.initial_state(p, seed=seed)
    m = ocn.Model(p)
    m.set(**st)
    o = oracle_mod.OracleModel(p)
    o.set(**st)
    o.project(1.0)
    return m, o


def test_qab2_fp64_taylor_green(oracle_mod):
    _, ocn = _gpu()
    p = inputs.config("taylor_green_32", timestepper="qab2")
    m, o = _pair(oracle_mod, ocn, p)
    m.time_step(p["dt"], p["steps"])
    o.time_step(p["dt"], p["steps"])
    _compare(m, o, p, True)


def test_qab2_fp32_cbl_100_steps(oracle_mod):
    _, ocn = _gpu()
    p = inputs.config("cbl_256", Nx=64, Ny=64, Nz=32, timestepper="qab2")
    m, o = _pair(oracle_mod, ocn, p)
    m.time_step(p["dt"], 100)
    o.time_step(p["dt"], 100)
    _compare(m, o, p, False)


@pytest.mark.parametrize("stepper", ["rk3", "qab2"])
@pytest.mark.parametrize("implicit", [False, True])
def test_vertical_diffusion_fp64(oracle_mod, stepper, implicit):
    _, ocn = _gpu()
    p = inputs.config("cbl_256", Nx=32, Ny=24, Nz=20, precision=64, timestepper=stepper)
    zf = np.asarray(p["z_faces"])
    rng = np.random.default_rng(3)
    p.update(nu_z=0.05 * np.exp(zf / 80.0) * (1 + 0.3 * rng.random(21)),
             kappa_z=0.08 * np.exp(zf / 60.0) * (1 + 0.3 * rng.random(21)), vertical_implicit=implicit)
    m, o = _pair(oracle_mod, ocn, p)
    dt = 20.0 if implicit else 2.0
    m.time_step(dt, 5)
    o.time_step(dt, 5)
    _compare(m, o, p, True)
    if not implicit:
        G = m.compute_tendencies()
        T = o.tendencies()
        for n in _fields(p):
            g, t = G[n].cpu().numpy(), T[n]
            assert np.abs(g - t).max() <= 1e-11 * np.abs(t).max(), n


def test_vertical_implicit_fp32_cbl_100_steps(oracle_mod):
    _, ocn = _gpu()
    p = inputs.config("cbl_256", Nx=64, Ny=64, Nz=32)
    zf = np.asarray(p["z_faces"])
    p.update(nu_z=1e-2 * np.exp(zf / 50.0), kappa_z=2e-2 * np.exp(zf / 50.0), vertical_implicit=True)
    m, o = _pair(oracle_mod, ocn, p)
    m.time_step(p["dt"], 100)
    o.time_step(p["dt"], 100)
    _compare(m, o, p, False)


def _tophat(ocn, oracle_mod, implicit, dt, steps):
    Nz = 20
    zf = np.linspace(-2.0, 2.0, Nz + 1)
    p = dict(Nx=4, Ny=4, Nz=Nz, Lx=1.0, Ly=1.0, z_faces=zf, precision=64, weno_order=5, closure="none",
             tracers=["b", "c"], eos="buoyancy_tracer", f=0.0, kappa_z=np.exp(-zf ** 2), vertical_implicit=implicit)
    zc = 0.5 * (zf[1:] + zf[:-1])
    c0 = np.broadcast_to(np.where(np.abs(zc) < 0.5, 1.0, 0.0)[:, None, None], (Nz, 4, 4)).copy()
    m = ocn.Model(p)
    m.set(c=c0)
    o = oracle_mod.OracleModel(p)
    o.set(c=c0)
    m.time_step(dt, steps)
    o.time_step(dt, steps)
    return m, o, p


def test_listing_top_hat_on_gpu(oracle_mod):
    """The paper's listing on the GPU: at dt = 0.5 the explicit step grows without bound (three
    steps already amplify the top hat by 1e6 or more), the implicit step stays within the initial
    range; both agree with the oracle."""
    _, ocn = _gpu()
    m, o, p = _tophat(ocn, oracle_mod, False, 0.5, 3)
    c = m.get_numpy("c")
    assert np.abs(c).max() > 1e3
    assert np.abs(c - o.get("c")).max() <= 1e-11 * np.abs(o.get("c")).max()
    m, o, p = _tophat(ocn, oracle_mod, True, 0.5, 20)
    c = m.get_numpy("c")
    assert c.max() <= 1.0 + 1e-12 and c.min() >= -1e-12
    assert np.abs(c - o.get("c")).max() <= 1e-11


def test_qab2_checkpoint_restart_bitwise():
    torch, ocn = _gpu()
    p = inputs.config("cbl_256", Nx=64, Ny=32, Nz=16, timestepper="qab2")
    st = inputs.initial_state(p)
    a = ocn.Model(p); a.set(**st); a.time_step(p["dt"], 6)
    b = ocn.Model(p); b.set(**st); b.time_step(p["dt"], 3)
    saved = b.checkpoint()
    del b
    c = ocn.Model(p)
    c.restore(saved)
    c.time_step(p["dt"], 3)
    for n in _fields(p):
        assert torch.equal(a.get(n), c.get(n)), n


def test_qab2_ensemble_matches_sequential():
    torch, ocn = _gpu()
    ps = [dict(q, timestepper="qab2") for q in inputs.ensemble_configs(n=3, sizes=(16, 24), depths=(8, 12))]
    E = ocn.Ensemble(ps)
    S = ocn.Ensemble(ps)
    S.set_mode(sequential=True)
    for i, q in enumerate(ps):
        st = inputs.initial_state(q, seed=inputs.SEED + i)
        E.members[i].set(**st)
        S.members[i].set(**st)
    E.time_step(5.0, 4)
    S.time_step(5.0, 4)
    for i in range(3):
        for n in ("u", "v", "w", "b"):
            assert torch.equal(E.members[i].get(n), S.members[i].get(n)), (i, n)


def test_stepper_and_diffusivity_argument_errors():
    _, ocn = _gpu()
    p = inputs.config("cbl_256", Nx=16, Ny=16, Nz=8)
    m = ocn.Model(p)
    with pytest.raises(ocn.OcnError):
        ocn._check(ocn.lib().ocn_set_time_stepper(m._h, 7, 0.1), "stepper")
    with pytest.raises(ocn.OcnError):
        m.set_vertical_diffusivity(nu=-1.0)
    with pytest.raises(ocn.OcnError):
        m.set_vertical_diffusivity(kappa=float("nan"))
