"""Batched ensembles: every kernel of the step is one launch over all members (a work list of
(member, block) pairs).  The arithmetic is the members' own, so batched stepping must equal
sequential stepping bit for bit, for uneven sizes, mixed schemes, tile variants and the learned
column closure, and the number of launches per step must not grow with the member count."""
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


def _pair(ocn, ps, seed0=inputs.SEED, setup=None):
    B = ocn.Ensemble(ps)
    B.set_mode("batched")
    S = ocn.Ensemble(ps)
    S.set_mode("sequential")
    for i, q in enumerate(ps):
        st = inputs.initial_state(q, seed=seed0 + i)
        for E in (B, S):
            E.members[i].set(**st)
            if setup:
                setup(E, i)
    return B, S


def _assert_equal(B, S, names=("u", "v", "w", "b")):
    torch = pytest.importorskip("torch")
    for i in range(len(B.members)):
        for n in names:
            assert torch.equal(B.members[i].get(n), S.members[i].get(n)), (i, n)


@pytest.mark.parametrize("precision,branches", [(32, 1), (32, 3), (64, 1)])
def test_batched_equals_sequential_uneven_sizes(ocn, precision, branches):
    ps = inputs.ensemble_configs(n=5, sizes=(16, 24, 32), depths=(8, 12, 16), precision=precision)
    B, S = _pair(ocn, ps)
    B.set_branches(branches)
    B.time_step(5.0, 3)
    S.time_step(5.0, 3)
    _assert_equal(B, S)
    # one batched launch per kernel of the step and branch: with one branch, the same count as
    # one member alone
    one = ocn.Ensemble(ps[:1])
    one.set_mode("concurrent")
    one.members[0].set(**inputs.initial_state(ps[0]))
    one.time_step(5.0, 1)
    assert B.launches_per_step() == branches * one.launches_per_step()


def test_batched_after_autotune_and_mixed_schemes(ocn):
    base = inputs.ensemble_configs(n=6, sizes=(16, 32), depths=(8, 16))
    zf = [np.asarray(q["z_faces"]) for q in base]
    ps = [dict(base[0]), dict(base[1], closure="smagorinsky"), dict(base[2], timestepper="qab2"),
          dict(base[3], nu_z=1e-2 * np.exp(zf[3] / 20.0), kappa_z=2e-2 * np.exp(zf[3] / 20.0),
               vertical_implicit=True),
          dict(base[4], nu_z=1e-3 * np.ones(len(zf[4])), kappa_z=1e-3 * np.ones(len(zf[4]))),
          dict(base[5])]
    B, S = _pair(ocn, ps)
    B.autotune()
    S.autotune()
    B.time_step(5.0, 2)
    S.time_step(5.0, 2)
    _assert_equal(B, S)
    # a second batched call replays the cached graph (QAB2 member now past its Euler start)
    B.time_step(5.0, 2)
    S.time_step(5.0, 2)
    _assert_equal(B, S)


def test_batched_learned_closure_shared_and_distinct_networks(ocn):
    ps = inputs.ensemble_configs(n=4, sizes=(16,), depths=(16,))
    nets = []
    for seed in (11, 12):
        net = ocn.MLP(inputs.MLP_SIZES, max_batch=1024)
        net.set_params(inputs.mlp_init(seed=seed))
        nets.append(net)
    mu = np.zeros(32)
    sigma = np.ones(32)
    sigma[:15] = 1e-5
    sigma[15:20] = (1e-8, 1e-4, 1e-5, 100.0, 10.0)

    def setup(E, i):
        # members 0, 1, 3 share network 0; member 2 has its own (a separate batched launch)
        # output scales per member (as with the buoyancy-flux-scaled closure)
        E.members[i].set_column_closure(nets[1 if i == 2 else 0], mu=mu, sigma=sigma,
                                        out_scale=(1e-6 * (i + 1), 1e-5, 1e-5), N2_background=ps[i]["N2"])

    B, S = _pair(ocn, ps, setup=setup)
    B.time_step(5.0, 3)
    S.time_step(5.0, 3)
    _assert_equal(B, S)
    for i in range(4):
        d = B.members[i].diagnostics()
        assert np.isfinite(d["max_div"])


def test_autotune_json_cache(ocn, tmp_path):
    cache = str(tmp_path / "tuning.json")
    ps = inputs.ensemble_configs(n=3, sizes=(16, 32), depths=(8, 16))
    E = ocn.Ensemble(ps)
    E.set_mode("batched")
    for i, q in enumerate(ps):
        E.members[i].set(**inputs.initial_state(q, seed=inputs.SEED + i))
    v1 = E.autotune(cache=cache)
    v2 = E.autotune(cache=cache)                # applied from the file, not re-timed
    assert v1 == v2 and all(0 <= x < ocn.TENDENCY_VARIANTS for x in v1)
    m = ocn.Model(ps[0])
    m.set(**inputs.initial_state(ps[0]))
    b1, ms1 = m.autotune(cache=cache)
    b2, ms2 = m.autotune(cache=cache)
    assert b1 == b2 and ms1 is not None and ms2 is None


def test_graph_caches_bounded_with_varying_dt(ocn):
    """Forty distinct time steps (each a new step graph) pass the cache bound; results equal direct launches."""
    torch = pytest.importorskip("torch")
    p = inputs.config("cbl_256", Nx=32, Ny=32, Nz=16)
    st = inputs.initial_state(p)
    a, b = ocn.Model(p), ocn.Model(p)
    a.set(**st)
    b.set(**st)
    b.set_option(ocn.OCN_OPT_GRAPHS, 0)
    ps = inputs.ensemble_configs(n=2, sizes=(16,), depths=(8,))
    E, S = _pair(ocn, ps)
    for i in range(40):
        dt = 2.0 + 0.05 * i
        a.time_step(dt, 1)
        b.time_step(dt, 1)
        E.time_step(dt, 1)
        S.time_step(dt, 1)
    for n in ("u", "v", "w", "b"):
        assert torch.equal(a.get(n), b.get(n)), n
    _assert_equal(E, S)
