"""ctypes wrapper around the FP64 CPU oracle (``oracle/ocn_oracle.c``).

ORACLE / TEST INFRASTRUCTURE.  Only the test suite, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import this module.  The CUDA
library and its Python binding never import it.

Parameters arrive as a plain ``dict`` (the same keys the tests hand to the CUDA
binding); nothing is shared with the CUDA path except the seeded input arrays.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "liboracle.so")
SRC = [os.path.join(HERE, "ocn_oracle.c")]
MAX_TRACERS = 4

CLOSURES = {"none": 0, "scalar": 1, "smagorinsky": 2, "amd": 3}
EOS = {"buoyancy_tracer": 0, "linear_ts": 1}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11 + OpenMP, IEEE arithmetic)."""
    os.makedirs(BUILD, exist_ok=True)
    newest = max(os.path.getmtime(p) for p in SRC + [os.path.join(HERE, "ocn_oracle.h"), os.path.join(HERE, "coeffs.h")])
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < newest:
        tmp = LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fopenmp", "-fPIC", "-shared", "-o", tmp] + SRC + ["-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, LIB)
    return LIB


class _Params(C.Structure):
    _fields_ = [
        ("Nx", C.c_int), ("Ny", C.c_int), ("Nz", C.c_int),
        ("Lx", C.c_double), ("Ly", C.c_double),
        ("zf", C.POINTER(C.c_double)),
        ("weno_order", C.c_int), ("closure", C.c_int),
        ("nu", C.c_double), ("kappa", C.c_double),
        ("Cs", C.c_double), ("Cb", C.c_double), ("Pr", C.c_double),
        ("C_amd", C.c_double),
        ("f", C.c_double),
        ("n_tracers", C.c_int), ("eos", C.c_int),
        ("g", C.c_double), ("alpha", C.c_double), ("beta", C.c_double), ("T0", C.c_double), ("S0", C.c_double),
        ("top_flux", C.c_double * (2 + MAX_TRACERS)),
        ("bottom_flux", C.c_double * (2 + MAX_TRACERS)),
        ("nthreads", C.c_int),
        ("timestepper", C.c_int), ("chi", C.c_double),
        ("nu_z", C.POINTER(C.c_double)), ("kappa_z", C.POINTER(C.c_double)), ("vertical_implicit", C.c_int),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        dp = C.POINTER(C.c_double)
        L.orc_create.restype = C.c_void_p
        L.orc_create.argtypes = [C.POINTER(_Params)]
        L.orc_destroy.argtypes = [C.c_void_p]
        L.orc_field_len.restype = C.c_size_t
        L.orc_field_len.argtypes = [C.c_void_p, C.c_int]
        L.orc_set.argtypes = [C.c_void_p, C.c_int, dp]
        L.orc_get.argtypes = [C.c_void_p, C.c_int, dp]
        L.orc_project.argtypes = [C.c_void_p, C.c_double]
        L.orc_time_step.argtypes = [C.c_void_p, C.c_double, C.c_int]
        L.orc_tendencies.argtypes = [C.c_void_p, dp, dp, dp, dp]
        L.orc_tendency_at.restype = C.c_double
        L.orc_tendency_at.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int]
        L.orc_diffusivity_at.restype = C.c_double
        L.orc_diffusivity_at.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int]
        L.orc_diagnostics.argtypes = [C.c_void_p, C.c_double, dp]
        L.orc_divergence.argtypes = [C.c_void_p, dp]
        L.orc_weno.restype = C.c_double
        L.orc_weno.argtypes = [dp, C.c_int, C.c_double]
        L.orc_weno_parts.argtypes = [dp, C.c_int, C.c_double, dp, dp]
        L.orc_centered.restype = C.c_double
        L.orc_centered.argtypes = [dp, C.c_int]
        L.orc_fft.argtypes = [dp, dp, C.c_int, C.c_int]
        L.orc_poisson.argtypes = [C.c_void_p, dp, dp]
        L.orc_grid_metrics.argtypes = [C.c_void_p, dp, dp, dp]
        L.orc_profiles.argtypes = [C.c_void_p, dp]
        L.orc_regrid.argtypes = [dp, C.c_int, dp, dp, C.c_int, dp]
        L.orc_closure_features.argtypes = [C.c_void_p, C.c_double, dp]
        L.orc_column_sgs_flux.argtypes = [C.c_void_p, dp]
        L.orc_coarse_grain.argtypes = [C.c_void_p, C.c_int, C.c_int, dp]
        L.orc_set_face_flux.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
        L.orc_set_face_diffusivity.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
        L.orc_vertical_diffusion.argtypes = [C.c_void_p, C.c_int, dp, dp, dp]
        L.orc_vertical_implicit_solve.argtypes = [C.c_void_p, C.c_int, dp, C.c_double, dp, dp]
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.POINTER(C.c_double))


# ---------------------------------------------------------------- building blocks
def weno(stencil, r: int, vel: float) -> float:
    s = np.ascontiguousarray(stencil, dtype=np.float64)
    assert s.size == 2 * r
    return lib().orc_weno(_dp(s), r, float(vel))


def weno_parts(stencil, r: int, vel: float):
    s = np.ascontiguousarray(stencil, dtype=np.float64)
    q = np.zeros(r); b = np.zeros(r)
    lib().orc_weno_parts(_dp(s), r, float(vel), _dp(q), _dp(b))
    return q, b


def centered(stencil, p: int) -> float:
    s = np.ascontiguousarray(stencil, dtype=np.float64)
    assert s.size == 2 * p
    return lib().orc_centered(_dp(s), p)


def fft(x: np.ndarray, sign: int = -1) -> np.ndarray:
    re = np.ascontiguousarray(np.real(x), dtype=np.float64).copy()
    im = np.ascontiguousarray(np.imag(x), dtype=np.float64).copy()
    lib().orc_fft(_dp(re), _dp(im), re.size, sign)
    return re + 1j * im


def regrid(zf_in, values, zf_out) -> np.ndarray:
    zi = np.ascontiguousarray(zf_in, dtype=np.float64); v = np.ascontiguousarray(values, dtype=np.float64)
    zo = np.ascontiguousarray(zf_out, dtype=np.float64); out = np.zeros(zo.size - 1)
    lib().orc_regrid(_dp(zi), v.size, _dp(v), _dp(zo), out.size, _dp(out))
    return out


NF = 32              # feature vector length of the learned column closure (20 used)
FACE_FLUX_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.POINTER(C.c_double))

# ---------------------------------------------------------------- model
FIELD_IDS = {"u": 0, "v": 1, "w": 2, "p": 10}


class OracleModel:
    """The FP64 oracle model.  ``params`` keys: Nx, Ny, Nz, Lx, Ly, z_faces,
    weno_order, closure, nu, kappa, Cs, Cb, Pr, C_amd, f, tracers (names),
    eos, g, alpha, beta, T0, S0, top_flux / bottom_flux (dicts by field name),
    nthreads."""

    def __init__(self, params: dict):
        p = dict(params)
        self.params = p
        self.Nx, self.Ny, self.Nz = int(p["Nx"]), int(p["Ny"]), int(p["Nz"])
        self.tracers = list(p.get("tracers", ["b"]))
        self._zf = np.ascontiguousarray(p["z_faces"], dtype=np.float64)
        assert self._zf.size == self.Nz + 1
        P = _Params()
        P.Nx, P.Ny, P.Nz = self.Nx, self.Ny, self.Nz
        P.Lx, P.Ly = float(p["Lx"]), float(p["Ly"])
        P.zf = _dp(self._zf)
        P.weno_order = int(p.get("weno_order", 5))
        P.closure = CLOSURES[p.get("closure", "none")]
        P.nu, P.kappa = float(p.get("nu", 0.0)), float(p.get("kappa", 0.0))
        P.Cs, P.Cb, P.Pr = float(p.get("Cs", 0.16)), float(p.get("Cb", 1.0)), float(p.get("Pr", 1.0))
        P.C_amd = float(p.get("C_amd", 1.0 / 12.0))
        P.f = float(p.get("f", 0.0))
        P.n_tracers = len(self.tracers)
        P.eos = EOS[p.get("eos", "buoyancy_tracer")]
        P.g, P.alpha, P.beta = float(p.get("g", 9.81)), float(p.get("alpha", 2e-4)), float(p.get("beta", 8e-4))
        P.T0, P.S0 = float(p.get("T0", 20.0)), float(p.get("S0", 35.0))
        names = ["u", "v"] + self.tracers
        for n, name in enumerate(names):
            P.top_flux[n] = float(p.get("top_flux", {}).get(name, 0.0))
            P.bottom_flux[n] = float(p.get("bottom_flux", {}).get(name, 0.0))
        P.nthreads = int(p.get("nthreads", 0))
        P.timestepper = {"rk3": 0, "qab2": 1}[p.get("timestepper", "rk3")]
        P.chi = float(p.get("chi", 0.1))
        self._nuz = self._kapz = None
        if p.get("nu_z") is not None:
            self._nuz = np.ascontiguousarray(np.broadcast_to(np.asarray(p["nu_z"], np.float64), (self.Nz + 1,)))
            P.nu_z = _dp(self._nuz)
        if p.get("kappa_z") is not None:
            self._kapz = np.ascontiguousarray(np.broadcast_to(np.asarray(p["kappa_z"], np.float64), (self.Nz + 1,)))
            P.kappa_z = _dp(self._kapz)
        P.vertical_implicit = int(bool(p.get("vertical_implicit", False)))
        self._P = P
        self._h = lib().orc_create(C.byref(P))
        if not self._h:
            raise ValueError("oracle rejected the parameters")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_destroy(h)
            self._h = None

    def fid(self, name: str) -> int:
        if name in FIELD_IDS:
            return FIELD_IDS[name]
        if name.startswith("G_"):
            return 20 + self.fid(name[2:])
        return 3 + self.tracers.index(name)

    def shape(self, name: str):
        base = name[2:] if name.startswith("G_") else name
        return (self.Nz + 1 if base == "w" else self.Nz, self.Ny, self.Nx)

    def set(self, **fields):
        for name, arr in fields.items():
            a = np.ascontiguousarray(arr, dtype=np.float64)
            assert a.shape == self.shape(name), (name, a.shape)
            lib().orc_set(self._h, self.fid(name), _dp(a))

    def get(self, name: str) -> np.ndarray:
        out = np.empty(self.shape(name), dtype=np.float64)
        lib().orc_get(self._h, self.fid(name), _dp(out))
        return out

    def project(self, dt_stage: float = 1.0):
        lib().orc_project(self._h, float(dt_stage))

    def time_step(self, dt: float, nsteps: int = 1):
        lib().orc_time_step(self._h, float(dt), int(nsteps))

    def tendencies(self):
        Nz, Ny, Nx = self.Nz, self.Ny, self.Nx
        Gu = np.empty((Nz, Ny, Nx)); Gv = np.empty((Nz, Ny, Nx)); Gw = np.empty((Nz + 1, Ny, Nx))
        Gc = np.empty((max(1, len(self.tracers)), Nz, Ny, Nx))
        lib().orc_tendencies(self._h, _dp(Gu), _dp(Gv), _dp(Gw), _dp(Gc))
        out = {"u": Gu, "v": Gv, "w": Gw}
        for n, t in enumerate(self.tracers):
            out[t] = Gc[n]
        return out

    def tendency_at(self, name: str, i: int, j: int, k: int) -> float:
        return lib().orc_tendency_at(self._h, self.fid(name), i, j, k)

    def diffusivity_at(self, which: int, i: int, j: int, k: int) -> float:
        return lib().orc_diffusivity_at(self._h, which, i, j, k)

    def divergence(self) -> np.ndarray:
        out = np.empty((self.Nz, self.Ny, self.Nx))
        lib().orc_divergence(self._h, _dp(out))
        return out

    def poisson(self, rhs: np.ndarray) -> np.ndarray:
        r = np.ascontiguousarray(rhs, dtype=np.float64)
        out = np.empty_like(r)
        lib().orc_poisson(self._h, _dp(r), _dp(out))
        return out

    def profiles(self) -> dict:
        """Horizontal means <b>, <u>, <v> at levels and total upward fluxes of b, u, v at faces."""
        Nz = self.Nz
        out = np.zeros(3 * Nz + 3 * (Nz + 1))
        lib().orc_profiles(self._h, _dp(out))
        F = out[3 * Nz:]
        return {"b": out[:Nz], "u": out[Nz:2 * Nz], "v": out[2 * Nz:3 * Nz],
                "Fb": F[:Nz + 1], "Fu": F[Nz + 1:2 * (Nz + 1)], "Fv": F[2 * (Nz + 1):]}

    def grid_metrics(self):
        zc = np.empty(self.Nz); dzc = np.empty(self.Nz); dzf = np.empty(self.Nz + 1)
        lib().orc_grid_metrics(self._h, _dp(zc), _dp(dzc), _dp(dzf))
        return zc, dzc, dzf

    def diagnostics(self, dt: float = 0.0) -> dict:
        nt = len(self.tracers)
        out = np.zeros(nt + 6)
        lib().orc_diagnostics(self._h, float(dt), _dp(out))
        d = {f"sum_{t}": out[n] for n, t in enumerate(self.tracers)}
        d.update(sum_u=out[nt], sum_v=out[nt + 1], sum_w=out[nt + 2], max_div=out[nt + 3], cfl=out[nt + 4],
                 nonfinite=int(out[nt + 5]))
        return d

    # ------------------------------------------------------------ learned column closure
    def closure_features(self, N2_background: float) -> np.ndarray:
        """Raw column features of every w-face, [(Nz+1)*Ny*Nx][NF] in (k, j, i) order."""
        X = np.zeros(((self.Nz + 1) * self.Ny * self.Nx, NF))
        lib().orc_closure_features(self._h, float(N2_background), _dp(X))
        return X

    def column_sgs_flux(self) -> np.ndarray:
        """The closure's vertical flux of b, ubar, vbar, [3][Nz+1][Ny][Nx]."""
        F = np.zeros((3, self.Nz + 1, self.Ny, self.Nx))
        lib().orc_column_sgs_flux(self._h, _dp(F))
        return F

    def coarse_grain(self, cx: int, cy: int) -> dict:
        """Box filter onto cx x cy columns: coarse u, v, w, b and subfilter fluxes tau [3][Nz+1][cy][cx]."""
        assert self.Nx % cx == 0 and self.Ny % cy == 0
        Nz = self.Nz
        n = cx * cy
        out = np.zeros(3 * Nz * n + (Nz + 1) * n + 3 * (Nz + 1) * n)
        lib().orc_coarse_grain(self._h, int(cx), int(cy), _dp(out))
        o = 0
        res = {}
        for name, levels in (("u", Nz), ("v", Nz), ("w", Nz + 1), ("b", Nz)):
            res[name] = out[o:o + levels * n].reshape(levels, cy, cx); o += levels * n
        res["tau"] = out[o:].reshape(3, Nz + 1, cy, cx)
        return res

    def set_face_flux(self, fn):
        """fn(model) -> F [3][Nz+1][Ny][Nx] called at every tendency evaluation (None removes it).
        Inside fn, ``model`` is this object with the stage state loaded."""
        if fn is None:
            lib().orc_set_face_flux(self._h, None, None)
            self._flux_cb = None
            return
        shape = (3, self.Nz + 1, self.Ny, self.Nx)

        def cb(ctx, h, F):
            out = np.ctypeslib.as_array(F, shape=shape)
            out[...] = fn(self)

        self._flux_cb = FACE_FLUX_FN(cb)
        lib().orc_set_face_flux(self._h, C.cast(self._flux_cb, C.c_void_p), None)

    def set_face_diffusivity(self, fn):
        """fn(model) -> K [3][Nz+1][Ny][Nx] (tracer and momentum diffusivities at every w-face of
        every column) called at the start of every stage; their horizontal means become that
        stage's implicit vertical diffusivity profiles.  None removes the hook."""
        if fn is None:
            lib().orc_set_face_diffusivity(self._h, None, None)
            self._diff_cb = None
            return
        shape = (3, self.Nz + 1, self.Ny, self.Nx)

        def cb(ctx, h, F):
            out = np.ctypeslib.as_array(F, shape=shape)
            out[...] = fn(self)

        self._diff_cb = FACE_FLUX_FN(cb)
        lib().orc_set_face_diffusivity(self._h, C.cast(self._diff_cb, C.c_void_p), None)

    def vertical_diffusion(self, q, kappa_faces, staggering: int = 0) -> np.ndarray:
        """D(q) = d/dz(kappa dq/dz) of one column (staggering 0: centres, 1: faces)."""
        q = np.ascontiguousarray(q, np.float64); kf = np.ascontiguousarray(kappa_faces, np.float64)
        out = np.zeros_like(q)
        lib().orc_vertical_diffusion(self._h, int(staggering), _dp(kf), _dp(q), _dp(out))
        return out

    def vertical_implicit_solve(self, rhs, kappa_faces, dtau: float, staggering: int = 0) -> np.ndarray:
        """q with (I - dtau D) q = rhs for one column."""
        r = np.ascontiguousarray(rhs, np.float64); kf = np.ascontiguousarray(kappa_faces, np.float64)
        out = np.zeros_like(r)
        lib().orc_vertical_implicit_solve(self._h, int(staggering), _dp(kf), float(dtau), _dp(r), _dp(out))
        return out
