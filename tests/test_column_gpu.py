"""GPU parity of the learned column closure against the FP64 oracle.

Tolerances (written here, derived from the arithmetic):
* features, closure fluxes, coarse-graining: FP32 state and FP32 arithmetic on short stencils;
  1e-5 of each quantity's largest magnitude (FP32 unit roundoff 6e-8 times the cancellation of
  a vertical difference of O(10^2) on these grids);
* learned fluxes: BF16 network, normwise 16 u_bf16 = 2^-5 per flux component (the network
  derivation of tests/test_mlp_gpu.py);
* tendency increment: the flux divergence is linear in F with operator norm <= 2 max(1/dz_c),
  so its error is bounded by that norm times the flux error bound;
* coupled steps: FP32 field tolerance 1e-4 plus four times the BF16 bound on the closure's
  own contribution to the state change.
"""
import numpy as np
import pytest

from oracle import mlp as omlp
from paper_2502_14148_gb300 import inputs

pytestmark = pytest.mark.gpu
TOL_BF16 = 16 * 2.0 ** -9


def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _params(Nx=32, Ny=24, Nz=20, **over):
    p = inputs.config("cbl_256", Nx=Nx, Ny=Ny, Nz=Nz)
    p.update(over)
    return p


def _state(p, oracle_mod, seed=3, amp=0.02):
    """A projected random state on top of the workload's stratification (oracle projection)."""
    st = inputs.initial_state(p, seed=seed)
    rnd = inputs.random_state(p, seed=seed + 1, amp=amp)
    o = oracle_mod.OracleModel(p)
    b = st["b"] + 1e-2 * p["N2"] * rnd["b"] * (p["Lz"] / p["Nz"])
    o.set(u=st["u"] + rnd["u"], v=st["v"] + rnd["v"], w=st["w"] + rnd["w"], b=b)
    o.project(1.0)
    return o, {n: o.get(n) for n in ("u", "v", "w", "b")}


def _gpu(p, fields):
    from paper_2502_14148_gb300 import ocn
    m = ocn.Model(p)
    m.set(project=False, **fields)
    return m


def _rel_max(a, b):
    a = np.asarray(a, np.float64); b = np.asarray(b, np.float64)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("shape", [(32, 24, 20), (12, 18, 4)])
def test_features_match_oracle(oracle_mod, shape):
    _need_gpu()
    p = _params(*shape)
    o, f = _state(p, oracle_mod)
    m = _gpu(p, f)
    N2 = p["N2"]
    Xg = m.closure_features(N2).cpu().numpy()
    Xo = o.closure_features(N2)
    for q in range(19):
        scale = max(np.abs(Xo[:, q]).max(), 1e-30)
        assert np.abs(Xg[:, q] - Xo[:, q]).max() <= 1e-5 * scale, q
    assert np.all(Xg[:, 20:] == 0)
    # the depth estimate sums Nz-1 FP32 terms (1 - g/N2) dz_f: bound 64 eps_32 sum (1 + |g|/N2) dz_f per column
    Nz, Ny, Nx = p["Nz"], p["Ny"], p["Nx"]
    zc = 0.5 * (np.asarray(p["z_faces"])[1:] + np.asarray(p["z_faces"])[:-1])
    dzf = np.r_[0.0, np.diff(zc), 0.0]
    g = Xo[:, 2].reshape(Nz + 1, Ny, Nx)
    bound = 64 * 2.0 ** -24 * ((1 + np.abs(g) / N2) * dzf[:, None, None]).sum(axis=0)
    err = np.abs(Xg[:, 19] - Xo[:, 19]).reshape(Nz + 1, Ny, Nx)
    assert np.all(err <= bound[None]), float((err / bound[None]).max())


def test_closure_fluxes_and_coarse_grain_match_oracle(oracle_mod):
    _need_gpu()
    p = _params(32, 24, 20)
    o, f = _state(p, oracle_mod)
    m = _gpu(p, f)
    Fg = m.column_fluxes().cpu().numpy()
    Fo = o.column_sgs_flux()
    for q in range(3):
        assert _rel_max(Fg[q], Fo[q]) < 1e-5, q
    for cx, cy in [(8, 6), (32, 24), (1, 1)]:
        cg = m.coarse_grain(cx, cy)
        co = o.coarse_grain(cx, cy)
        for name in ("u", "v", "w", "b"):
            # scale by the fine field: box means of w over wide boxes are near zero
            scale = max(np.abs(f[name]).max(), 1e-300)
            assert np.abs(cg[name].cpu().numpy() - co[name]).max() < 1e-5 * scale, (cx, name)
        for q in range(3):
            assert _rel_max(cg["tau"][q].cpu().numpy(), co["tau"][q]) < 1e-5, (cx, q)


def _normalisation(X):
    """Feature means and scales; a feature that is constant over the samples (Jb, f, N2 of one
    model) is scaled by its magnitude so that rounding of the mean cannot blow it up."""
    mu = np.zeros(32); sigma = np.ones(32)
    mu[:20] = X[:, :20].mean(axis=0)
    sd = X[:, :20].std(axis=0)
    const = sd <= 1e-6 * np.abs(mu[:20])
    sigma[:20] = np.where(const, np.maximum(np.abs(mu[:20]), 1e-30), np.where(sd > 0, sd, 1.0))
    return mu, sigma


def _network(X, seed=11):
    from paper_2502_14148_gb300 import ocn
    params = inputs.mlp_init(seed=seed)
    net = ocn.MLP(inputs.MLP_SIZES, max_batch=1024)
    net.set_params(params)
    params32 = [(W.astype(np.float32).astype(np.float64), b.astype(np.float32).astype(np.float64)) for W, b in params]
    mu, sigma = _normalisation(X)
    mu = mu.astype(np.float32).astype(np.float64)
    sigma = sigma.astype(np.float32).astype(np.float64)
    return net, params32, mu, sigma


SCALE = np.array([1e-6, 1e-4, 1e-4])


@pytest.mark.parametrize("shape", [(32, 24, 20), (12, 18, 4)])
def test_learned_flux_matches_oracle(oracle_mod, shape):
    _need_gpu()
    p = _params(*shape)
    o, f = _state(p, oracle_mod)
    m = _gpu(p, f)
    X = o.closure_features(p["N2"])
    net, params, mu, sigma = _network(X)
    m.set_column_closure(net, mu, sigma, SCALE, p["N2"])
    Fg = m.column_fluxes(learned=True).cpu().numpy()
    Fo = omlp.closure_fluxes(params, X, mu, sigma, SCALE, (p["Nz"] + 1, p["Ny"], p["Nx"]))
    assert np.all(Fg[:, 0] == 0) and np.all(Fg[:, -1] == 0)
    for q in range(3):
        err = np.linalg.norm(Fg[q] - Fo[q]) / np.linalg.norm(Fo[q])
        assert err < TOL_BF16, (q, err)


def test_tendency_increment_matches_oracle(oracle_mod):
    _need_gpu()
    p = _params(32, 24, 20)
    o, f = _state(p, oracle_mod)
    m = _gpu(p, f)
    X = o.closure_features(p["N2"])
    net, params, mu, sigma = _network(X)
    G0 = m.compute_tendencies()
    m.set_column_closure(net, mu, sigma, SCALE, p["N2"])
    G1 = m.compute_tendencies()
    T0 = o.tendencies()
    shape = (p["Nz"] + 1, p["Ny"], p["Nx"])
    o.set_face_flux(lambda mod: omlp.closure_fluxes(params, mod.closure_features(p["N2"]), mu, sigma, SCALE, shape))
    T1 = o.tendencies()
    o.set_face_flux(None)
    Fo = omlp.closure_fluxes(params, X, mu, sigma, SCALE, shape)
    rdz = 1.0 / np.diff(np.asarray(p["z_faces"])).min()
    for q, name in enumerate(("b", "u", "v")):
        dg = (G1[name] - G0[name]).cpu().numpy().astype(np.float64)
        do = T1[name] - T0[name]
        bound = TOL_BF16 * 2 * rdz * np.linalg.norm(Fo[q])
        assert np.linalg.norm(dg - do) <= bound, (name, np.linalg.norm(dg - do), bound)
        assert np.linalg.norm(do) > 0
    # w is untouched by the column closure
    assert np.array_equal(G1["w"].cpu().numpy(), G0["w"].cpu().numpy())


def test_coupled_steps_match_oracle(oracle_mod):
    _need_gpu()
    p = _params(32, 24, 20)
    o, f = _state(p, oracle_mod)
    X = o.closure_features(p["N2"])
    net, params, mu, sigma = _network(X)
    scale = np.array([1e-6, 3e-4, 3e-4])
    shape = (p["Nz"] + 1, p["Ny"], p["Nx"])
    dt, n = 5.0, 3
    o_plain = oracle_mod.OracleModel(p)
    o_plain.set(**f)
    o_plain.time_step(dt, n)
    o.set_face_flux(lambda mod: omlp.closure_fluxes(params, mod.closure_features(p["N2"]), mu, sigma, scale, shape))
    o.time_step(dt, n)
    m = _gpu(p, f)
    m.set_column_closure(net, mu, sigma, scale, p["N2"])
    m.time_step(dt, n)
    m.synchronize()
    assert m.diagnostics()["status"] == "OK"
    for name in ("u", "v", "w", "b"):
        g = m.get_numpy(name).astype(np.float64)
        ref, plain = o.get(name), o_plain.get(name)
        effect = np.linalg.norm(ref - plain)
        err = np.linalg.norm(g - ref)
        bound = 1e-4 * np.linalg.norm(ref) + 4 * TOL_BF16 * effect
        assert err <= bound, (name, err, bound, effect)


def test_coupled_steps_diffusivity_mode_match_oracle(oracle_mod):
    """The closure in diffusivity form: per stage, the column means of max(0, scale y) at each face
    become the implicit vertical diffusivity profiles (kappa: tracers, nu: momentum).  The oracle
    does the same with its FP64 network through its diffusivity hook."""
    _need_gpu()
    p = _params(32, 24, 20)
    o, f = _state(p, oracle_mod)
    X = o.closure_features(p["N2"])
    net, params, mu, sigma = _network(X)
    scale = np.array([0.05, 0.02, 0.0])                 # m^2/s per unit network output
    shape = (p["Nz"] + 1, p["Ny"], p["Nx"])
    dt, n = 5.0, 3
    o_plain = oracle_mod.OracleModel(p)
    o_plain.set(**f)
    o_plain.time_step(dt, n)
    o.set_face_diffusivity(lambda mod: omlp.closure_diffusivities(params, mod.closure_features(p["N2"]), mu, sigma,
                                                                  scale, shape))
    o.time_step(dt, n)
    m = _gpu(p, f)
    m.set_column_closure(net, mu, sigma, scale, p["N2"], mode="diffusivity")
    m.time_step(dt, n)
    m.synchronize()
    assert m.diagnostics()["status"] == "OK"
    moved = 0
    for name in ("u", "v", "w", "b"):
        g = m.get_numpy(name).astype(np.float64)
        ref, plain = o.get(name), o_plain.get(name)
        effect = np.linalg.norm(ref - plain)
        moved += effect > 1e-3 * np.linalg.norm(ref - np.mean(ref))
        err = np.linalg.norm(g - ref)
        bound = 1e-4 * np.linalg.norm(ref) + 4 * TOL_BF16 * effect
        assert err <= bound, (name, err, bound, effect)
    assert moved >= 2                                   # the closure changed the state measurably
    # a tendency evaluation takes nothing from an implicit closure
    G0 = _gpu(p, f).compute_tendencies()
    m2 = _gpu(p, f)
    m2.set_column_closure(net, mu, sigma, scale, p["N2"], mode="diffusivity")
    G1 = m2.compute_tendencies()
    for name in G0:
        assert np.array_equal(G0[name].cpu().numpy(), G1[name].cpu().numpy()), name


def test_diffusivity_mode_batched_ensemble_equals_single_models(oracle_mod):
    torch = _need_gpu()
    from paper_2502_14148_gb300 import ocn
    ps = [_params(16, 16, 12, top_flux={"b": 1e-8}), _params(24, 24, 16, top_flux={"b": 5e-8}, f=0.0)]
    states = [_state(p, oracle_mod, seed=11 + i)[1] for i, p in enumerate(ps)]
    X = oracle_mod.OracleModel(ps[0])
    X.set(**states[0])
    net, params, mu, sigma = _network(X.closure_features(ps[0]["N2"]))
    scale = (0.05, 0.02, 0.0)
    ens = ocn.Ensemble(ps)
    ens.set_mode("batched")
    singles = []
    for p, st, mem in zip(ps, states, ens.members):
        mem.set(project=False, **st)
        mem.set_column_closure(net, mu, sigma, scale, p["N2"], mode="diffusivity")
        s_ = _gpu(p, st)
        s_.set_column_closure(net, mu, sigma, scale, p["N2"], mode="diffusivity")
        singles.append(s_)
    ens.time_step(5.0, 3)
    ens.synchronize()
    for s_ in singles:
        s_.time_step(5.0, 3)
        s_.synchronize()
    for mem, s_ in zip(ens.members, singles):
        for name in ("u", "v", "w", "b"):
            assert torch.equal(mem.get(name), s_.get(name)), name


def test_diffusivity_mode_validation():
    _need_gpu()
    from paper_2502_14148_gb300 import ocn
    p = _params(16, 16, 8)
    m = ocn.Model(p)
    net = ocn.MLP(inputs.MLP_SIZES, max_batch=256)
    with pytest.raises(ocn.OcnError) as ei:
        ocn._check(ocn.lib().ocn_set_column_closure_mode(m._h, 2), "ocn_set_column_closure_mode")
    assert ei.value.status == -1
    m.set_vertical_diffusivity(np.full(9, 1e-3), np.full(9, 1e-3), implicit=True)
    with pytest.raises(ocn.OcnError) as ei:            # the model's own profiles come first
        m.set_column_closure(net, mode="diffusivity")
    assert ei.value.status == -8
    q = inputs.config("les_512", Nx=16, Ny=16, Nz=8)       # not a buoyancy-tracer model
    with pytest.raises(ocn.OcnError) as ei:
        ocn.Model(q).set_column_closure(None, mode="diffusivity")
    assert ei.value.status == -7


def test_ensemble_members_with_closure_match_single_models(oracle_mod):
    torch = _need_gpu()
    from paper_2502_14148_gb300 import ocn
    ps = [_params(16, 16, 12, top_flux={"b": 1e-8}), _params(24, 24, 16, top_flux={"b": 5e-8}, f=0.0)]
    states = [_state(p, oracle_mod, seed=7 + i)[1] for i, p in enumerate(ps)]
    X = oracle_mod.OracleModel(ps[0])
    X.set(**states[0])
    net, params, mu, sigma = _network(X.closure_features(ps[0]["N2"]))
    ens = ocn.Ensemble(ps)
    singles = []
    for p, st, mem in zip(ps, states, ens.members):
        mem.set(project=False, **st)
        mem.set_column_closure(net, mu, sigma, SCALE, p["N2"])
        s = _gpu(p, st)
        s.set_column_closure(net, mu, sigma, SCALE, p["N2"])
        singles.append(s)
    ens.time_step(5.0, 3)
    ens.synchronize()
    for s in singles:
        s.time_step(5.0, 3)
        s.synchronize()
    for mem, s in zip(ens.members, singles):
        for name in ("u", "v", "w", "b"):
            assert torch.equal(mem.get(name), s.get(name)), name
    # removing the closure restores the plain model exactly
    p = ps[0]
    a = _gpu(p, states[0]); b = _gpu(p, states[0])
    a.set_column_closure(net, mu, sigma, SCALE, p["N2"]); a.set_column_closure(None)
    a.time_step(5.0, 2); b.time_step(5.0, 2)
    assert torch.equal(a.get("b"), b.get("b"))


def test_column_closure_rejects_unsupported_models():
    _need_gpu()
    from paper_2502_14148_gb300 import ocn
    p = inputs.config("les_512", Nx=16, Ny=16, Nz=8)      # linear T,S equation of state
    m = ocn.Model(p)
    net = ocn.MLP(inputs.MLP_SIZES, max_batch=256)
    with pytest.raises(ocn.OcnError) as ei:
        m.set_column_closure(net)
    assert ei.value.status == -7
    p2 = _params(16, 16, 8)
    m2 = ocn.Model(p2)
    small = ocn.MLP((32, 64, 16), max_batch=256)
    with pytest.raises(ocn.OcnError) as ei:
        m2.set_column_closure(small)
    assert ei.value.status == -7
    with pytest.raises(ocn.OcnError):
        m2.set_column_closure(net, sigma=np.zeros(32))
