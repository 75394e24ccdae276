"""Pins of the oracle's learned-column-closure pieces: features, closure fluxes, box
coarse-graining and the face-flux hook, against closed forms, exact properties and
hand-computed cases."""
import numpy as np
import pytest

from oracle import mlp as omlp
from paper_2502_14148_gb300 import inputs


def _model(oracle_mod, Nx=8, Ny=6, Nz=10, closure="none", stretch=True, **kw):
    Lz = 20.0
    zf = inputs.tanh_faces(Nz, Lz, 1.5) if stretch else inputs.uniform_faces(Nz, Lz)
    p = dict(Nx=Nx, Ny=Ny, Nz=Nz, Lx=16.0, Ly=12.0, z_faces=zf, weno_order=5, closure=closure,
             tracers=["b"], eos="buoyancy_tracer", f=1e-4, top_flux={"b": 3e-8}, nu=1e-3, kappa=2e-3)
    p.update(kw)
    return oracle_mod.OracleModel(p), p


def _centres(p):
    zf = np.asarray(p["z_faces"])
    return zf, 0.5 * (zf[1:] + zf[:-1])


def test_features_linear_stratification(oracle_mod):
    m, p = _model(oracle_mod)
    zf, zc = _centres(p)
    Nx, Ny, Nz = p["Nx"], p["Ny"], p["Nz"]
    N2 = 1e-5
    m.set(b=np.broadcast_to(N2 * zc[:, None, None], (Nz, Ny, Nx)).copy())
    X = m.closure_features(N2).reshape(Nz + 1, Ny, Nx, -1)
    for k in range(Nz + 1):
        x = X[k, 2, 3]
        for mm in range(-2, 3):
            q = k + mm
            expect = N2 if 1 <= q <= Nz - 1 else 0.0
            assert abs(x[mm + 2] - expect) < 1e-12 * N2 * 1e3, (k, mm)
        assert np.all(x[5:15] == 0.0)
        assert x[15] == 3e-8 and x[16] == 1e-4 and x[17] == N2
        assert abs(x[18] - (zf[-1] - zf[k])) < 1e-12
        assert abs(x[19]) < 1e-9            # no deficit: h = 0
        assert np.all(x[20:] == 0.0)
    # half the background stratification: deficit 1/2 on every interior face
    X2 = m.closure_features(2 * N2).reshape(Nz + 1, Ny, Nx, -1)
    assert abs(X2[0, 0, 0, 19] - 0.5 * (zc[-1] - zc[0])) < 1e-10


def test_features_mixed_layer_depth(oracle_mod):
    """b = N2 min(z, -h_m): the estimate is h_m minus the half-thickness of the top cell."""
    m, p = _model(oracle_mod, Nz=16, stretch=False)
    zf, zc = _centres(p)
    Nx, Ny, Nz = p["Nx"], p["Ny"], p["Nz"]
    N2, h_m = 2e-5, 7.3
    b = N2 * np.minimum(zc, -h_m)
    m.set(b=np.broadcast_to(b[:, None, None], (Nz, Ny, Nx)).copy())
    X = m.closure_features(N2).reshape(Nz + 1, Ny, Nx, -1)
    assert abs(X[0, 0, 0, 19] - (h_m - (zf[-1] - zc[-1]))) < 1e-10
    # gradient features around the mixed-layer base, face by face (stencil order k-2..k+2)
    dzf = np.r_[0.0, np.diff(zc), 0.0]
    kb = int(np.searchsorted(zc, -h_m))                 # first centre above the base
    for k in (kb - 1, kb, kb + 1, kb + 2):
        for mm in range(-2, 3):
            q = k + mm
            expect = (b[q] - b[q - 1]) / dzf[q] if 1 <= q <= Nz - 1 else 0.0
            assert abs(X[k, 1, 1, mm + 2] - expect) < 1e-15 + 1e-12 * N2, (k, mm)


def test_features_velocity_gradients_and_stencil_order(oracle_mod):
    m, p = _model(oracle_mod)
    zf, zc = _centres(p)
    Nx, Ny, Nz = p["Nx"], p["Ny"], p["Nz"]
    dzf = np.r_[0.0, np.diff(zc), 0.0]
    u = np.broadcast_to((0.3 * zc ** 2)[:, None, None], (Nz, Ny, Nx)).copy()
    v = np.broadcast_to((-0.2 * zc)[:, None, None], (Nz, Ny, Nx)).copy()
    m.set(u=u, v=v, b=np.zeros((Nz, Ny, Nx)))
    X = m.closure_features(1e-5).reshape(Nz + 1, Ny, Nx, -1)
    k = 5
    for mm in range(-2, 3):
        q = k + mm
        assert abs(X[k, 0, 0, 5 + mm + 2] - 0.3 * (zc[q] ** 2 - zc[q - 1] ** 2) / dzf[q]) < 1e-12
        assert abs(X[k, 0, 0, 10 + mm + 2] + 0.2) < 1e-12


def test_column_sgs_flux_scalar_closed_form(oracle_mod):
    m, p = _model(oracle_mod, closure="scalar")
    zf, zc = _centres(p)
    Nx, Ny, Nz = p["Nx"], p["Ny"], p["Nz"]
    N2 = 1e-5
    u = np.broadcast_to((0.1 * zc)[:, None, None], (Nz, Ny, Nx)).copy()
    m.set(u=u, b=np.broadcast_to(N2 * zc[:, None, None], (Nz, Ny, Nx)).copy())
    F = m.column_sgs_flux()
    assert np.all(F[:, 0] == 0) and np.all(F[:, -1] == 0)
    np.testing.assert_allclose(F[0, 1:-1], -2e-3 * N2, rtol=1e-10)
    np.testing.assert_allclose(F[1, 1:-1], -1e-3 * 0.1, rtol=1e-10)
    assert np.all(F[2] == 0)


def _random_divfree(m, p, seed=5):
    st = inputs.random_state(p, seed=seed)
    m.set(u=st["u"], v=st["v"], w=st["w"], b=st["b"])
    m.project(1.0)
    return m


def test_coarse_grain_identity_and_divergence_free(oracle_mod):
    m, p = _model(oracle_mod, closure="scalar")
    _random_divfree(m, p)
    Nx, Ny, Nz = p["Nx"], p["Ny"], p["Nz"]
    c = m.coarse_grain(Nx, Ny)                       # box of one column: the identity
    for name in ("u", "v", "w", "b"):
        np.testing.assert_array_equal(c[name], m.get(name))
    np.testing.assert_allclose(c["tau"], m.column_sgs_flux(), rtol=1e-13, atol=1e-18)
    # face-average restriction keeps the discrete velocity divergence-free on the coarse grid
    cx, cy = Nx // 2, Ny // 3
    c = m.coarse_grain(cx, cy)
    zf = np.asarray(p["z_faces"])
    dzc = np.diff(zf)
    dX, dY = p["Lx"] / cx, p["Ly"] / cy
    div = (np.roll(c["u"], -1, 2) - c["u"]) / dX + (np.roll(c["v"], -1, 1) - c["v"]) / dY \
        + (c["w"][1:] - c["w"][:-1]) / dzc[:, None, None]
    scale = np.abs(c["w"]).max() / dzc.min()
    assert np.abs(div).max() < 1e-12 * scale


def test_coarse_grain_hand_computed_flux(oracle_mod):
    """Four fine columns into one: tau_b at face 1 = <w b_f> - <w><b_f> by hand."""
    m, p = _model(oracle_mod, Nx=2, Ny=2, Nz=3, stretch=False)
    w = np.zeros((4, 2, 2)); w[1] = [[1.0, 2.0], [3.0, 6.0]]
    b = np.zeros((3, 2, 2)); b[1] = [[2.0, 4.0], [6.0, 8.0]]
    m.set(w=w, b=b)
    c = m.coarse_grain(1, 1)
    # b_f at face 1 = (b0 + b1)/2 = [1, 2, 3, 4]; <w b_f> = 38/4; <w> = 3; <b_f> = 5/2
    assert abs(c["tau"][0, 1, 0, 0] - 2.0) < 1e-14
    assert c["tau"][0, 0, 0, 0] == 0.0 and c["tau"][0, 3, 0, 0] == 0.0
    assert abs(c["w"][1, 0, 0] - 3.0) < 1e-15 and abs(c["b"][1, 0, 0] - 5.0) < 1e-15


def test_coarse_grain_box_constant_tracer_has_no_subfilter_flux(oracle_mod):
    m, p = _model(oracle_mod)
    _random_divfree(m, p)
    Nx, Ny, Nz = p["Nx"], p["Ny"], p["Nz"]
    rng = np.random.default_rng(2)
    coarse = rng.standard_normal((Nz, Ny // 2, Nx // 2))
    m.set(b=np.repeat(np.repeat(coarse, 2, axis=1), 2, axis=2))
    c = m.coarse_grain(Nx // 2, Ny // 2)
    assert np.abs(c["tau"][0]).max() < 1e-14 * np.abs(m.get("w")).max() * np.abs(coarse).max() * 10


def _tend(m):
    return m.tendencies()


def test_face_flux_hook_linear_flux_closed_form(oracle_mod):
    m, p = _model(oracle_mod, closure="scalar")
    _random_divfree(m, p)
    Nx, Ny, Nz = p["Nx"], p["Ny"], p["Nz"]
    zf = np.asarray(p["z_faces"]); dzc = np.diff(zf)
    G0 = _tend(m)
    a = 2.5e-3
    F = np.zeros((3, Nz + 1, Ny, Nx))
    F[0] = a * zf[:, None, None]
    F[1] = np.arange(Nx)[None, None, :] * 1e-3        # depends on i only: tests the u-face average
    F[2] = np.arange(Ny)[None, :, None] * 2e-3        # depends on j only: tests the v-face average
    m.set_face_flux(lambda model: F)
    G1 = _tend(m)
    m.set_face_flux(None)
    dGb = G1["b"] - G0["b"]
    np.testing.assert_allclose(dGb[1:-1], -a, rtol=1e-9)
    np.testing.assert_allclose(dGb[0], -a * zf[1] / dzc[0], rtol=1e-9)
    np.testing.assert_allclose(dGb[-1], a * zf[-2] / dzc[-1], rtol=1e-9)
    # u column at face i gets F averaged over columns i-1, i: (i - 1/2) 1e-3, wrapping at i = 0
    fu = 0.5 * (np.roll(np.arange(Nx), 1) + np.arange(Nx)) * 1e-3
    dGu = G1["u"] - G0["u"]
    np.testing.assert_allclose(dGu[0], np.broadcast_to(-fu / dzc[0], (Ny, Nx)), rtol=1e-9)
    np.testing.assert_allclose(dGu[-1], np.broadcast_to(fu / dzc[-1], (Ny, Nx)), rtol=1e-9)
    assert np.abs(dGu[1:-1]).max() < 1e-12
    fv = 0.5 * (np.roll(np.arange(Ny), 1) + np.arange(Ny)) * 2e-3
    dGv = G1["v"] - G0["v"]
    np.testing.assert_allclose(dGv[0], np.broadcast_to((-fv / dzc[0])[:, None], (Ny, Nx)), rtol=1e-9)
    assert np.abs(dGv[1:-1]).max() < 1e-12


def test_face_flux_hook_conserves_column_integrals(oracle_mod):
    m, p = _model(oracle_mod)
    _random_divfree(m, p)
    Nx, Ny, Nz = p["Nx"], p["Ny"], p["Nz"]
    dzc = np.diff(np.asarray(p["z_faces"]))
    G0 = _tend(m)
    F = np.random.default_rng(4).standard_normal((3, Nz + 1, Ny, Nx))
    m.set_face_flux(lambda model: F)
    G1 = _tend(m)
    m.set_face_flux(None)
    for name in ("b", "u", "v"):
        col = ((G1[name] - G0[name]) * dzc[:, None, None]).sum(axis=0)
        assert np.abs(col).max() < 1e-12 * np.abs(F).max() * 10, name


def test_closure_fluxes_linear_network_and_walls():
    rng = np.random.default_rng(9)
    W = rng.standard_normal((16, 32)); b = rng.standard_normal(16)
    X = rng.standard_normal((5 * 2 * 3, 32))
    mu, sigma = rng.standard_normal(32), 1.0 + rng.random(32)
    scale = np.array([2.0, 3.0, 5.0])
    F = omlp.closure_fluxes([(W, b)], X, mu, sigma, scale, (5, 2, 3))
    y = ((X - mu) / sigma) @ W.T + b
    for q in range(3):
        expect = scale[q] * y[:, q].reshape(5, 2, 3)
        expect[0] = 0; expect[-1] = 0
        np.testing.assert_allclose(F[q], expect, rtol=1e-14)


def test_face_diffusivity_hook_equals_implicit_profiles(oracle_mod):
    """The diffusivity hook's column means become the implicit profiles of every stage: per-column
    diffusivities kappa_k (1 + r_ij), nu_k (1 - r_ij) with sum_ij r_ij = 0 step exactly like a model
    given the profiles kappa, nu directly (pinned in tests/test_timestep_oracle.py), for RK3 and
    QAB2; the hook sees each stage's initial state (three calls per RK3 step, the first with the
    state the step starts from)."""
    Nz, Ny, Nx = 10, 6, 8
    zf = inputs.tanh_faces(Nz, 20.0, 1.5)
    kap = 0.2 * np.exp(zf / 8.0); kap[0] = kap[-1] = 0.0
    nu = 0.1 * np.exp(zf / 5.0); nu[0] = nu[-1] = 0.0
    r = np.random.default_rng(8).standard_normal((Ny, Nx)) * 0.3
    r -= r.mean()
    K = np.zeros((3, Nz + 1, Ny, Nx))
    K[0] = kap[:, None, None] * (1.0 + r)
    K[1] = nu[:, None, None] * (1.0 - r)
    for stepper in ("rk3", "qab2"):
        m, p = _model(oracle_mod, closure="amd", timestepper=stepper)
        _random_divfree(m, p)
        st = {n: m.get(n) for n in ("u", "v", "w", "b")}
        seen = []

        def hook(model):
            seen.append(model.get("b").copy())
            return K
        m.set_face_diffusivity(hook)
        m.time_step(7.0, 2)
        ref, _ = _model(oracle_mod, closure="amd", timestepper=stepper, kappa_z=kap, nu_z=nu, vertical_implicit=True)
        ref.set(**st)
        ref.time_step(7.0, 2)
        for n in ("u", "v", "w", "b"):
            a, b = m.get(n), ref.get(n)
            assert np.abs(a - b).max() <= 1e-13 * np.abs(b).max(), (stepper, n)
        assert len(seen) == (6 if stepper == "rk3" else 2)
        assert np.array_equal(seen[0], st["b"])
        # the diffusion acted: the run differs from one without it
        plain, _ = _model(oracle_mod, closure="amd", timestepper=stepper)
        plain.set(**st)
        plain.time_step(7.0, 2)
        assert np.abs(plain.get("b") - m.get("b")).max() > 1e-6 * np.abs(m.get("b")).max()


def test_closure_diffusivities_relu_and_walls():
    rng = np.random.default_rng(10)
    W = rng.standard_normal((16, 32)); b = rng.standard_normal(16)
    X = rng.standard_normal((5 * 2 * 3, 32))
    mu, sigma = rng.standard_normal(32), 1.0 + rng.random(32)
    scale = np.array([2.0, 3.0, 5.0])
    K = omlp.closure_diffusivities([(W, b)], X, mu, sigma, scale, (5, 2, 3))
    y = ((X - mu) / sigma) @ W.T + b
    for q in range(2):
        expect = np.maximum(scale[q] * y[:, q].reshape(5, 2, 3), 0.0)
        expect[0] = 0; expect[-1] = 0
        np.testing.assert_allclose(K[q], expect, rtol=1e-14)
    assert (K[:2] >= 0).all() and (K[:2] == 0).any() and (K[2] == 0).all()
