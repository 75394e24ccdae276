"""Pins of the oracle's QAB2 stepper (Eq. qab2) and vertical diffusion, explicit or semi-implicit
(Eqs. tracer-with-tendency, tracer-time-discretization, predictor-velocity)."""
import math

import numpy as np
import pytest

from paper_2502_14148_gb300 import inputs


def _column_model(oracle_mod, Nz=20, stretch=False, **kw):
    zf = inputs.tanh_faces(Nz, 4.0, 1.5) - 0.0 if stretch else np.linspace(-2.0, 2.0, Nz + 1)
    if stretch:
        zf = zf + 2.0 - zf[-1]                 # keep the top at z = 2
    p = dict(Nx=4, Ny=4, Nz=Nz, Lx=1.0, Ly=1.0, z_faces=zf, weno_order=5, closure="none",
             tracers=["b", "c"], eos="buoyancy_tracer", f=0.0)
    p.update(kw)
    return oracle_mod.OracleModel(p), p


def _metrics(p):
    zf = np.asarray(p["z_faces"])
    zc = 0.5 * (zf[1:] + zf[:-1])
    return zf, zc, np.diff(zf), np.r_[0.0, np.diff(zc), 0.0]


def test_vertical_operator_exact_conservative_symmetric(oracle_mod):
    m, p = _column_model(oracle_mod, Nz=12)
    zf, zc, dzc, dzf = _metrics(p)
    kap = 0.3 * np.ones(13)
    # second-order finite volumes are exact for quadratics in the interior (uniform grid)
    D = m.vertical_diffusion(zc ** 2, kap)
    np.testing.assert_allclose(D[1:-1], 2 * 0.3, rtol=1e-12)
    rng = np.random.default_rng(1)
    for stretch in (False, True):
        m, p = _column_model(oracle_mod, Nz=12, stretch=stretch)
        zf, zc, dzc, dzf = _metrics(p)
        kf = np.exp(-rng.random(13))
        # centres: no flux through the walls -> conservative; symmetric, negative semi-definite in the dz_c product
        q, r = rng.standard_normal(12), rng.standard_normal(12)
        Dq, Dr = m.vertical_diffusion(q, kf), m.vertical_diffusion(r, kf)
        assert abs((dzc * Dq).sum()) < 1e-13 * np.abs(Dq).max()
        assert abs((dzc * r * Dq).sum() - (dzc * q * Dr).sum()) < 1e-12 * np.abs(dzc * r * Dq).sum()
        assert (dzc * q * Dq).sum() < 0
        # faces (walls held at 0): symmetric, negative definite in the dz_f product over the interior faces
        w, s = rng.standard_normal(13), rng.standard_normal(13)
        w[0] = w[-1] = s[0] = s[-1] = 0.0
        Dw, Ds = m.vertical_diffusion(w, kf, 1), m.vertical_diffusion(s, kf, 1)
        assert Dw[0] == 0 and Dw[-1] == 0
        assert abs((dzf * s * Dw).sum() - (dzf * w * Ds).sum()) < 1e-12 * np.abs(dzf * s * Dw).sum()
        assert (dzf * w * Dw).sum() < 0


def test_implicit_solve_against_dense_and_eigenmode(oracle_mod):
    rng = np.random.default_rng(2)
    for stag in (0, 1):
        m, p = _column_model(oracle_mod, Nz=10, stretch=True)
        n = 10 + stag
        kf = np.exp(-rng.random(11))
        # assemble D column by column from the operator, then solve densely
        A = np.zeros((n, n))
        for j in range(n):
            e = np.zeros(n); e[j] = 1.0
            A[:, j] = m.vertical_diffusion(e, kf, stag)
        rhs = rng.standard_normal(n)
        if stag:
            rhs[0] = rhs[-1] = 0.0
        dtau = 0.7
        q = m.vertical_implicit_solve(rhs, kf, dtau, stag)
        sl = slice(1, n - 1) if stag else slice(0, n)
        M = np.eye(n) - dtau * A
        ref = np.linalg.solve(M[sl, sl], rhs[sl])
        np.testing.assert_allclose(q[sl], ref, rtol=1e-12, atol=1e-14)
    # discrete cosine eigenmode (constant kappa, uniform grid): one step multiplies it by 1/(1 + dtau lambda)
    m, p = _column_model(oracle_mod, Nz=16)
    zf, zc, dzc, dzf = _metrics(p)
    kap, dz, mode = 0.2, dzc[0], 3
    q0 = np.cos(math.pi * mode * (zc - zf[0]) / (zf[-1] - zf[0]))
    lam = kap * (2 * math.sin(math.pi * mode / (2 * 16)) / dz) ** 2
    q1 = m.vertical_implicit_solve(q0, kap * np.ones(17), 0.9)
    np.testing.assert_allclose(q1, q0 / (1 + 0.9 * lam), rtol=1e-12, atol=1e-14)


def _tophat_run(oracle_mod, dt, t_end, implicit):
    Nz = 20
    zf = np.linspace(-2.0, 2.0, Nz + 1)
    kap = np.exp(-zf ** 2)                          # the paper's listing: kappa(z) = exp(-z^2)
    m, p = _column_model(oracle_mod, Nz=Nz, kappa_z=kap, vertical_implicit=implicit)
    zc = 0.5 * (zf[1:] + zf[:-1])
    c0 = np.where(np.abs(zc) < 0.5, 1.0, 0.0)
    m.set(c=np.broadcast_to(c0[:, None, None], (Nz, 4, 4)).copy())
    m.time_step(dt, int(round(t_end / dt)))
    return m.get("c")[:, 0, 0], c0


def test_listing_top_hat_diffusivity_explicit_vs_implicit(oracle_mod):
    """The paper's time-discretization listing: with dt = 0.5 the explicit step is unstable, the
    vertically implicit one stable; a short explicit step agrees with the implicit solution."""
    with np.errstate(all="ignore"):
        ex, c0 = _tophat_run(oracle_mod, 0.5, 10.0, implicit=False)
    assert not np.all(np.isfinite(ex)) or np.abs(ex).max() > 1e3
    im, _ = _tophat_run(oracle_mod, 0.5, 10.0, implicit=True)
    assert np.abs(im).max() <= 1.0 + 1e-12 and im.min() >= -1e-12       # maximum principle
    ref, _ = _tophat_run(oracle_mod, 1e-2, 10.0, implicit=False)
    assert np.abs(im - ref).max() < 0.01
    fine, _ = _tophat_run(oracle_mod, 1e-2, 10.0, implicit=True)
    assert np.abs(fine - ref).max() < np.abs(im - ref).max() / 5        # the implicit error shrinks with dt
    # the column integral is conserved (no flux through the walls)
    assert abs(im.sum() - c0.sum()) < 1e-12 * c0.sum()


def _inertial(oracle_mod, dt, chi, t_end):
    f = 1e-4
    p = dict(Nx=4, Ny=4, Nz=4, Lx=1.0, Ly=1.0, z_faces=np.linspace(-1, 0, 5), weno_order=5, closure="none",
             tracers=["b"], eos="buoyancy_tracer", f=f, timestepper="qab2", chi=chi)
    m = oracle_mod.OracleModel(p)
    m.set(u=np.ones((4, 4, 4)), v=np.zeros((4, 4, 4)))
    m.time_step(dt, int(round(t_end / dt)))
    t = t_end
    return math.hypot(m.get("u")[0, 0, 0] - math.cos(f * t), m.get("v")[0, 0, 0] + math.sin(f * t))


def test_qab2_convergence_orders():
    """QAB2 is formally first order for chi = 0.1 and second order (AB2) for chi = 0."""
    import oracle.oracle as oracle_mod
    T = 2 * math.pi / 1e-4 / 4
    e1 = [_inertial(oracle_mod, T / n, 0.1, T) for n in (50, 100)]
    e2 = [_inertial(oracle_mod, T / n, 0.0, T) for n in (50, 100)]
    assert 1.7 < e1[0] / e1[1] < 2.3, e1
    assert 3.4 < e2[0] / e2[1] < 4.6, e2


def test_qab2_first_step_is_forward_euler(oracle_mod):
    p = inputs.config("taylor_green_32", Nx=16, Ny=16, Nz=16)
    p.update(timestepper="qab2")
    st = inputs.initial_state(p)
    m = oracle_mod.OracleModel(p)
    m.set(**st)
    m.project(1.0)
    u0 = {k: m.get(k) for k in ("u", "v", "w", "b")}
    G = m.tendencies()
    dt = 0.05
    e = oracle_mod.OracleModel(dict(p, timestepper="rk3"))
    e.set(**{k: u0[k] + dt * G[k] for k in u0})
    e.project(dt)
    m.set(**u0)                                   # setting fields restarts QAB2 with an Euler step
    m.time_step(dt, 1)
    for k in ("u", "v", "w", "b"):
        np.testing.assert_allclose(m.get(k), e.get(k), rtol=0, atol=1e-13 * max(1.0, np.abs(u0[k]).max()))


def test_qab2_conserves_tracers_and_momentum(oracle_mod):
    p = inputs.config("taylor_green_32", Nx=16, Ny=16, Nz=16)
    p.update(timestepper="qab2", N2=0.0)
    st = inputs.initial_state(p)
    m = oracle_mod.OracleModel(p)
    m.set(**st)
    m.project(1.0)
    d0 = m.diagnostics()
    m.time_step(0.02, 10)
    d1 = m.diagnostics()
    for k in ("sum_b", "sum_u", "sum_v"):
        assert abs(d1[k] - d0[k]) < 1e-12 * max(1.0, abs(d0[k])), k
    assert d1["max_div"] < 1e-10
