"""Seeded synthetic inputs: grids, workload parameter sets and initial states.

This module holds no arithmetic of the method.  It only states the workloads
(grid sizes, physical constants, forcing) and draws their initial conditions;
both the CUDA binding and the test oracle consume what it returns.  All noise is
drawn from numpy's counter-based Philox generator keyed by (seed, field).

Workloads (synthetic LES stand-ins shaped after the paper's Eady LES listing,
Sec. 3.1.3, and the convective / wind-driven boundary-layer set-ups):

* ``taylor_green_32``: 32^3, L = 2 pi, FP64, WENO5, nu = kappa = 1e-3,
  buoyancy tracer b = 0.01 z, Taylor-Green velocity + N(0, 1e-3) noise.
* ``cbl_256``: convective boundary layer 256x256x128, 512 m x 512 m x 256 m,
  tanh-stretched z (sigma = 1.5, refined at the surface), WENO5, AMD,
  f = 1e-4, surface buoyancy flux 1e-8 m^2 s^-3, N^2 = 1e-5, noise 1e-3.
* ``les_512``: wind- and convection-driven LES 512x512x256 at 1 m spacing,
  WENO9, Smagorinsky-Lilly, T and S with a linear EOS, f = 1e-4, surface
  stress -1e-4 m^2 s^-2 on u, surface T flux 5.1e-6 K m s^-1, noise 1e-3.
Any of them can be re-sized (``Nx=..`` etc.) keeping the grid spacing.
"""
from __future__ import annotations

import math

import numpy as np

SEED = 20250220


def uniform_faces(Nz: int, Lz: float) -> np.ndarray:
    """Nz+1 equally spaced face heights from -Lz to 0."""
    return np.linspace(-Lz, 0.0, Nz + 1)


def tanh_faces(Nz: int, Lz: float, sigma: float = 1.5) -> np.ndarray:
    """Face heights z_k = -Lz (1 - tanh(sigma k / Nz) / tanh(sigma)), k = 0..Nz:
    fine spacing at the surface, coarse at the bottom."""
    k = np.arange(Nz + 1, dtype=np.float64)
    z = -Lz * (1.0 - np.tanh(sigma * k / Nz) / math.tanh(sigma))
    z[0], z[-1] = -Lz, 0.0
    return z


def config(name: str, **over) -> dict:
    """Parameter dict of a named workload; keyword overrides re-size it (the
    horizontal spacing and, for uniform z, the vertical spacing are kept)."""
    if name == "taylor_green_32":
        p = dict(Nx=32, Ny=32, Nz=32, Lx=2 * math.pi, Ly=2 * math.pi, Lz=2 * math.pi, stretch=None,
                 precision=64, weno_order=5, closure="scalar", nu=1e-3, kappa=1e-3, f=0.0,
                 tracers=["b"], eos="buoyancy_tracer", dt=1e-2, steps=20,
                 init="taylor_green", N2=0.01, noise=1e-3)
        dx = None
    elif name == "cbl_256":
        p = dict(Nx=256, Ny=256, Nz=128, Lx=512.0, Ly=512.0, Lz=256.0, stretch=1.5,
                 precision=32, weno_order=5, closure="amd", C_amd=1.0 / 12.0, f=1e-4,
                 tracers=["b"], eos="buoyancy_tracer", top_flux={"b": 1e-8}, dt=10.0, steps=1000,
                 init="stratified", N2=1e-5, noise=1e-3)
        dx = 2.0
    elif name == "les_512":
        p = dict(Nx=512, Ny=512, Nz=256, Lx=512.0, Ly=512.0, Lz=256.0, stretch=None,
                 precision=32, weno_order=9, closure="smagorinsky", Cs=0.16, Cb=1.0, Pr=1.0, f=1e-4,
                 tracers=["T", "S"], eos="linear_ts", g=9.81, alpha=2e-4, beta=8e-4, T0=20.0, S0=35.0,
                 top_flux={"u": -1e-4, "T": 5.1e-6}, dt=2.0, steps=200,
                 init="stratified", N2=1e-5, noise=1e-3)
        dx = 1.0
    else:
        raise KeyError(name)
    p["name"] = name
    for key in ("Nx", "Ny", "Nz"):
        if key in over and dx is not None:
            L = {"Nx": "Lx", "Ny": "Ly", "Nz": "Lz"}[key]
            if key != "Nz" or p["stretch"] is None:
                p[L] = p[L] * over[key] / p[key]
    p.update(over)
    if p.get("stretch"):
        p["z_faces"] = tanh_faces(p["Nz"], p["Lz"], p["stretch"])
    else:
        p["z_faces"] = uniform_faces(p["Nz"], p["Lz"])
    p.setdefault("top_flux", {})
    p.setdefault("bottom_flux", {})
    return p


def ensemble_configs(n: int = 64, seed: int = SEED, sizes=(64, 96, 128), depths=(64, 80, 96), spacing: float = 2.0,
                     precision: int = 32, dt: float = 5.0) -> list:
    """Convective-boundary-layer ensemble: members of uneven sizes (Nx = Ny from `sizes`, Nz from
    `depths`, horizontal spacing and mean vertical spacing `spacing` m, tanh-stretched z) with
    surface buoyancy flux log-uniform in [1e-9, 1e-7] m^2 s^-3, N^2 log-uniform in [1e-6, 1e-4] s^-2
    and f uniform in [0, 1.4e-4] s^-1; WENO5, AMD, seeded noise 1e-3."""
    g = np.random.Generator(np.random.Philox(key=[seed, 999]))
    out = []
    for i in range(n):
        N = int(sizes[int(g.integers(len(sizes)))])
        Nz = int(depths[int(g.integers(len(depths)))])
        Jb = float(np.exp(g.uniform(np.log(1e-9), np.log(1e-7))))
        N2 = float(np.exp(g.uniform(np.log(1e-6), np.log(1e-4))))
        f = float(g.uniform(0.0, 1.4e-4))
        p = dict(name=f"cbl_member_{i}", Nx=N, Ny=N, Nz=Nz, Lx=spacing * N, Ly=spacing * N, Lz=spacing * Nz,
                 stretch=1.5, precision=precision, weno_order=5, closure="amd", C_amd=1.0 / 12.0, f=f,
                 tracers=["b"], eos="buoyancy_tracer", top_flux={"b": Jb}, bottom_flux={}, dt=dt,
                 init="stratified", N2=N2, noise=1e-3, member=i)
        p["z_faces"] = tanh_faces(Nz, p["Lz"], 1.5)
        out.append(p)
    return out


MLP_SIZES = (32, 128, 128, 128, 16)


def mlp_init(seed: int = SEED, sizes=MLP_SIZES) -> list:
    """Seeded initial weights of the column-closure network: W_l ~ N(0, 1/n_in), b_l = 0."""
    out = []
    for l in range(len(sizes) - 1):
        g = np.random.Generator(np.random.Philox(key=[seed, 500 + l]))
        W = g.standard_normal((sizes[l + 1], sizes[l])) / math.sqrt(sizes[l])
        out.append((W, np.zeros(sizes[l + 1])))
    return out


def mlp_batch(seed: int, M: int, n_in: int = 32, n_out: int = 16, n_real_in: int = 17, n_real_out: int = 3):
    """A seeded synthetic batch (features zero-padded to n_in, targets to n_out) for kernel tests."""
    g = np.random.Generator(np.random.Philox(key=[seed, 600]))
    X = np.zeros((M, n_in)); X[:, :n_real_in] = g.standard_normal((M, n_real_in))
    T = np.zeros((M, n_out)); T[:, :n_real_out] = g.standard_normal((M, n_real_out))
    mask = np.zeros(n_out); mask[:n_real_out] = 1.0
    return X, T, mask


def _normal(seed: int, field: int, shape) -> np.ndarray:
    g = np.random.Generator(np.random.Philox(key=[seed, field]))
    return g.standard_normal(size=shape)


def positions(p: dict):
    """Cell-centre and face coordinates of the grid (x, y uniform; z from z_faces)."""
    Nx, Ny = p["Nx"], p["Ny"]
    dx, dy = p["Lx"] / Nx, p["Ly"] / Ny
    xf = dx * np.arange(Nx)
    yf = dy * np.arange(Ny)
    zf = np.asarray(p["z_faces"], dtype=np.float64)
    return xf, xf + 0.5 * dx, yf, yf + 0.5 * dy, zf, 0.5 * (zf[1:] + zf[:-1])


def initial_state(p: dict, seed: int = SEED) -> dict:
    """Seeded FP64 initial fields in the [z][y][x] layout (w has Nz+1 levels)."""
    Nx, Ny, Nz = p["Nx"], p["Ny"], p["Nz"]
    xf, xc, yf, yc, zf, zc = positions(p)
    u = np.zeros((Nz, Ny, Nx)); v = np.zeros((Nz, Ny, Nx)); w = np.zeros((Nz + 1, Ny, Nx))
    out = {}
    init = p.get("init", "rest")
    if init == "taylor_green":
        Z, Y, X = np.meshgrid(zc, yc, xf, indexing="ij")
        u = np.sin(X) * np.cos(Y) * np.cos(Z)
        Z, Y, X = np.meshgrid(zc, yf, xc, indexing="ij")
        v = -np.cos(X) * np.sin(Y) * np.cos(Z)
        b = p.get("N2", 0.0) * np.broadcast_to(zc[:, None, None], (Nz, Ny, Nx))
        out["b"] = np.array(b)
    elif init == "taylor_green_2d":
        Z, Y, X = np.meshgrid(zc, yc, xf, indexing="ij")
        u = np.sin(X) * np.cos(Y)
        Z, Y, X = np.meshgrid(zc, yf, xc, indexing="ij")
        v = -np.cos(X) * np.sin(Y)
        out["b"] = np.array(np.broadcast_to(p.get("N2", 0.0) * zc[:, None, None], (Nz, Ny, Nx)))
    elif init in ("stratified", "rest"):
        N2 = p.get("N2", 0.0) if init == "stratified" else 0.0
        prof = np.broadcast_to(zc[:, None, None], (Nz, Ny, Nx))
        if p.get("eos", "buoyancy_tracer") == "linear_ts":
            out["T"] = np.array(p.get("T0", 20.0) + N2 * prof / (p.get("g", 9.81) * p.get("alpha", 2e-4)))
            out["S"] = np.full((Nz, Ny, Nx), p.get("S0", 35.0))
        else:
            out["b"] = np.array(N2 * prof)
    else:
        raise KeyError(init)
    amp = p.get("noise", 0.0)
    if amp:
        u = u + amp * _normal(seed, 0, u.shape)
        v = v + amp * _normal(seed, 1, v.shape)
        w = w + amp * _normal(seed, 2, w.shape)
    w[0] = 0.0
    w[-1] = 0.0
    out.update(u=np.ascontiguousarray(u), v=np.ascontiguousarray(v), w=np.ascontiguousarray(w))
    for t in p.get("tracers", []):
        out.setdefault(t, np.zeros((Nz, Ny, Nx)))
    return out


def random_state(p: dict, seed: int = SEED, amp: float = 1.0) -> dict:
    """Unstructured random fields (for operator-level parity checks)."""
    Nx, Ny, Nz = p["Nx"], p["Ny"], p["Nz"]
    out = {
        "u": amp * _normal(seed, 10, (Nz, Ny, Nx)),
        "v": amp * _normal(seed, 11, (Nz, Ny, Nx)),
        "w": amp * _normal(seed, 12, (Nz + 1, Ny, Nx)),
    }
    out["w"][0] = 0.0
    out["w"][-1] = 0.0
    for n, t in enumerate(p.get("tracers", [])):
        out[t] = _normal(seed, 20 + n, (Nz, Ny, Nx))
    return out
