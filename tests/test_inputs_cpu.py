"""The seeded synthetic inputs against the recipe they state: grid sizes and spacings of the named
workloads, the tanh-stretched vertical grid (surface refinement of the convective boundary layer),
the initial stratification, the noise amplitude and its seeding, and the ensemble's forcing ranges."""
import math

import numpy as np

from paper_2502_14148_gb300 import inputs


def test_named_workloads_shapes_and_spacing():
    les = inputs.config("les_512")
    assert (les["Nx"], les["Ny"], les["Nz"]) == (512, 512, 256)
    assert np.allclose(np.diff(les["z_faces"]), 1.0) and les["Lx"] / les["Nx"] == 1.0
    cbl = inputs.config("cbl_256")
    assert (cbl["Nx"], cbl["Ny"], cbl["Nz"]) == (256, 256, 128) and cbl["Lx"] / cbl["Nx"] == 2.0
    tg = inputs.config("taylor_green_32")
    assert tg["Lx"] == 2 * math.pi and tg["precision"] == 64
    # resized: horizontal spacing kept, uniform vertical spacing kept
    small = inputs.config("les_512", Nx=128, Ny=64, Nz=32)
    assert small["Lx"] / small["Nx"] == 1.0 and small["Ly"] / small["Ny"] == 1.0
    assert np.allclose(np.diff(small["z_faces"]), 1.0)


def test_tanh_grid_refines_at_the_surface():
    zf = inputs.config("cbl_256")["z_faces"]
    dz = np.diff(zf)
    assert zf[0] == -256.0 and zf[-1] == 0.0 and np.all(dz > 0)
    assert np.all(np.diff(dz) < 0)                      # monotonically finer toward the surface
    # z_k = -Lz (1 - tanh(s k / N) / tanh s): the spacing tends to dz/dk = Lz s sech^2(s k / N) / (N tanh s),
    # Lz s sech^2(s) / (N tanh s) at the surface and Lz s / (N tanh s) at the bottom (within the variation of
    # dz/dk over one cell, about 1 %)
    s, N, L = 1.5, 128, 256.0
    assert abs(dz[-1] - L * s / (N * math.tanh(s) * math.cosh(s) ** 2)) < 0.02 * dz[-1]
    assert abs(dz[0] - L * s / (N * math.tanh(s))) < 0.02 * dz[0]
    assert 0.55 < dz[-1] < 0.65 and 3.2 < dz[0] < 3.4     # about 0.6 m at the top, 3.3 m at the bottom


def test_initial_states_are_seeded_and_stratified():
    p = inputs.config("cbl_256", Nx=32, Ny=32, Nz=16)
    a, b = inputs.initial_state(p), inputs.initial_state(p)
    c = inputs.initial_state(p, seed=inputs.SEED + 1)
    for name in ("u", "v", "w", "b"):
        assert np.array_equal(a[name], b[name]), name
    assert not np.array_equal(a["u"], c["u"])
    assert np.all(a["w"][0] == 0) and np.all(a["w"][-1] == 0)   # impenetrable walls
    assert abs(a["u"].std() - 1e-3) < 1e-4 and abs(a["u"].mean()) < 1e-4
    zc = 0.5 * (p["z_faces"][1:] + p["z_faces"][:-1])
    assert np.allclose(a["b"], p["N2"] * zc[:, None, None])
    les = inputs.config("les_512", Nx=16, Ny=16, Nz=8)
    s = inputs.initial_state(les)
    zc = 0.5 * (les["z_faces"][1:] + les["z_faces"][:-1])
    # T from N^2 = g alpha dT/dz, S uniform
    assert np.allclose(s["T"], 20.0 + 1e-5 * zc[:, None, None] / (9.81 * 2e-4)) and np.all(s["S"] == 35.0)


def test_ensemble_forcing_ranges_and_seeding():
    ms = inputs.ensemble_configs(n=64)
    key = lambda m: (m["Nx"], m["Nz"], m["top_flux"]["b"], m["N2"], m["f"])
    assert [key(m) for m in ms] == [key(m) for m in inputs.ensemble_configs(n=64)]          # seeded
    assert [key(m) for m in ms] != [key(m) for m in inputs.ensemble_configs(n=64, seed=1)]
    assert {m["Nx"] for m in ms} <= {64, 96, 128} and {m["Nz"] for m in ms} <= {64, 80, 96}
    assert len({m["Nx"] for m in ms}) == 3 and len({m["Nz"] for m in ms}) == 3        # uneven members
    jb = np.array([m["top_flux"]["b"] for m in ms])
    n2 = np.array([m["N2"] for m in ms])
    f = np.array([m["f"] for m in ms])
    assert jb.min() >= 1e-9 and jb.max() <= 1e-7 and n2.min() >= 1e-6 and n2.max() <= 1e-4
    assert f.min() >= 0.0 and f.max() <= 1.4e-4
    # log-uniform: the logs spread over the range rather than clustering at the top
    assert np.log10(jb).std() > 0.4 and np.log10(n2).std() > 0.4
    for m in ms:
        assert m["Lx"] / m["Nx"] == 2.0 and abs(m["z_faces"][-1]) < 1e-12 and m["z_faces"][0] == -2.0 * m["Nz"]
