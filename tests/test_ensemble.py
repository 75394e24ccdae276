"""Ensembles (uneven members stepped together), coarse-graining profiles and conservative regridding."""
import numpy as np
import pytest

from paper_2502_14148_gb300 import inputs


def test_library_regrid_matches_oracle(oracle_mod):
    """Host-side conservative regridding of the library against the oracle's (no GPU needed)."""
    from paper_2502_14148_gb300 import build, ocn
    build.build()
    rng = np.random.default_rng(3)
    zi = inputs.tanh_faces(96, 192.0)
    vals = rng.standard_normal(96)
    for zo in (inputs.tanh_faces(64, 192.0), inputs.uniform_faces(16, 192.0), zi):
        np.testing.assert_allclose(ocn.regrid(zi, vals, zo), oracle_mod.regrid(zi, vals, zo), rtol=1e-13, atol=1e-15)


@pytest.fixture(scope="module")
def ocn():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_14148_gb300 import build, ocn as mod
    build.build()
    return mod


def _members(precision, n=3):
    ps = inputs.ensemble_configs(n=n, sizes=(16, 24, 32), depths=(8, 12, 16), precision=precision, dt=5.0)
    return ps


@pytest.mark.gpu
def test_profiles_parity_fp64(ocn, oracle_mod):
    for p in _members(64, n=2):
        st = inputs.initial_state(p, seed=inputs.SEED + p["member"])
        g = ocn.Model(p); g.set(**st); g.time_step(p["dt"], 3)
        o = oracle_mod.OracleModel(p); o.set(**st); o.project(1.0); o.time_step(p["dt"], 3)
        pg, po = g.profiles(), o.profiles()
        for key in ("b", "u", "v", "Fb", "Fu", "Fv"):
            scale = max(np.abs(po[key]).max(), 1e-300)
            assert np.abs(pg[key] - po[key]).max() / scale < 1e-10, key


@pytest.mark.gpu
@pytest.mark.parametrize("precision", [64, 32])
def test_ensemble_matches_members_and_oracle(ocn, oracle_mod, precision):
    ps = _members(precision)
    E = ocn.Ensemble(ps)
    S = ocn.Ensemble(ps)
    S.set_mode(sequential=True)
    states = []
    for i, p in enumerate(ps):
        st = inputs.initial_state(p, seed=inputs.SEED + i)
        if precision == 32:
            st = {k: x.astype(np.float32).astype(np.float64) for k, x in st.items()}
        states.append(st)
        E.members[i].set(**st)
        S.members[i].set(**st)
    E.autotune()
    E.time_step(5.0, 3)
    S.time_step(5.0, 3)
    assert E.launches_per_step() > 0
    for i, p in enumerate(ps):
        o = oracle_mod.OracleModel(p); o.set(**states[i]); o.project(1.0); o.time_step(5.0, 3)
        for name in ("u", "v", "w", "b"):
            a = E.members[i].get_numpy(name)
            assert np.array_equal(a, S.members[i].get_numpy(name)), (i, name)   # concurrent == sequential
            ref = o.get(name)
            if precision == 64:
                assert np.abs(a - ref).max() / np.abs(ref).max() < 1e-11, (i, name)
            else:
                assert np.linalg.norm(a - ref) / np.linalg.norm(ref) < 1e-4, (i, name)
